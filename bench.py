#!/usr/bin/env python3
"""RMTR seconds per load step on the 3D 129^3 four-level workload (20
penny-shaped fractures, pressure ramp p_t = 5e-4 t, t = 1..10), plus the
Hessian-vector product's throughput and roofline, on one GB300.

One "step" is one pseudo-time load step: pressure_set + rmtr_load_step (all
of the hot path: energy, gradient, hessvec, projected CG, TR control,
transfers, coarse feasible set, level model, V-cycles).  Run step k solves
ramp step t = (k - 1) mod 10 + 1 and restarts from the fractured state at
t = 1, so every timed pressure lies on the 10-step ramp to 5e-3.  Inputs are
seeded synthetic fracture networks (no dataset); the state lives in HBM.

By default the line also carries the metric's comparison, measured in the
same run: the same ramp steps from the same warmed state in plain FP64
(plain start) and in mixed precision with the plain start, with the per-field
error of the mixed fields against the FP64 fields at every step; and the
FP64 oracle timed on the host cores (whole load steps of the same workload
eight times coarser per axis, beside the GPU on those same steps).

  python bench.py [--steps K] [--warmup W] [--precision fp64|mixed]
  python bench.py --impl reference      # the FP64 CPU oracle

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
# The same workload eight times coarser per axis (four levels 3^3 -> 17^3, the
# same 20 discs, material and ramp): the size on which the FP64 oracle runs
# whole load steps in seconds, timed beside the GPU on equal work.
WORKLOAD_SMALL = dict(WORKLOAD, workload="3d_17^3_q1_4level_20discs_ramp", n_coarse=[3, 3, 3],
                      h_coarse=0.5)
# The pressure ramp of the 3D workload: p_t = 5e-4 t for t = 1 .. 10 (final
# 5e-3).  Step k of a run (warm-up and timed steps counted together from 1)
# is ramp step t = (k - 1) mod 10 + 1; at t = 1 the state restarts from the
# fractured initial state, so no pressure above 5e-3 is ever solved.
RAMP = 10
# The paper's own 3D scenario at its own size (Sec. 5.2, three-dimensional
# scenarios): unit cube, 50^3 coarse grid and four levels (393^3 nodes,
# 242,793,828 dofs), 100 fractures as rectangular plates, granite-like
# lambda = mu = 1e5 (E = 2.5e5, nu = 0.25), G_c = 1, clamped boundary, and
# the pressure p_k = p0 + k dt p_c with p0 = 0.01, dt = 0.05, p_c = 1.
PAPER_SCALE = {
    "workload": "3d_393^3_q1_4level_100plates_paper", "dim": 3, "n_coarse": [50, 50, 50],
    "levels": 4, "h_coarse": 1.0 / 49, "E": 2.5e5, "nu": 0.25, "Gc": 1.0, "ls_over_h": 2.0,
    "fractures": 100, "seed": PI.SEED_3D_PAPER, "p0": 0.01, "dp": 0.05,
}
METRIC = "RMTR s/load-step & hessvec GDoF/s: mixed+learned vs FP64 plain, same GB300"

# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per launch of the
# roofline kernels on this workload, from one ncu capture of
# `bench.py --kernels-only`; to be re-captured whenever those kernels change.
TRAFFIC_HESSVEC_FP32 = (69.044e6 + 17.576e6) + (47.787e6 + 1.250e6)  # element pass + gather
TRAFFIC_HESSVEC_FP64 = 7595.291e6 + 86.475e6
UNIT = "s/load-step"
# FP32 flops of one element of the 3D FP32 Hessian product (the paired-FMA
# element algebra and its corner sums), from the FP32 instruction counts of
# one ncu capture (FFMA2 x4, FFMA x2, FADD2/FMUL2 x2, FADD/FMUL x1): 6,135 M
# flop over the 144^3 element evaluations of an owner-computes launch.
FLOP32_PER_ELEMENT = 2055
# FP32 lanes per SM (Blackwell): the ALU roofline is SMs x lanes x 2 flop
# (one FMA) x the SM clock sampled while the kernels ran.
FP32_LANES_PER_SM = 128


def ramp_t(k: int) -> int:
    """Ramp step (1 .. RAMP) of run step k (1-based)."""
    return (k - 1) % RAMP + 1


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["fp64", "mixed"], default="mixed")
    ap.add_argument("--start", choices=["plain", "extrapolate"], default="extrapolate",
                    help="starting iterate of each load step (plain = x_{t-1})")
    ap.add_argument("--no-compare", action="store_true",
                    help="skip the FP64-plain and plain-start arms (run by default)")
    ap.add_argument("--compare-fp64", action="store_true",
                    help="accepted for old command lines; the comparison runs by default")
    ap.add_argument("--oracle-worker", default=None, help=argparse.SUPPRESS)
    ap.add_argument("--kernels-only", action="store_true",
                    help="set up the workload state, launch the element kernels and exit")
    ap.add_argument("--coarse-n", type=int, default=17,
                    help="coarsest nodes per axis (17 = the 129^3 workload)")
    ap.add_argument("--coarse-model", choices=["first_order", "galerkin"], default="first_order")
    ap.add_argument("--batched", action="store_true",
                    help="the uneven 2D batch (64 instances, 129^2 .. 1025^2) instead of the 3D workload")
    ap.add_argument("--batch-threads", type=int, default=0)
    ap.add_argument("--batched-ops", action="store_true",
                    help="time only the batched operators (one persistent launch over the instances)")
    ap.add_argument("--batch-count", type=int, default=64, help="--batched-ops: instances of the draw")
    ap.add_argument("--batch-bps", type=int, default=0,
                    help="--batched-ops: blocks per SM of the product launch (0: autotune)")
    ap.add_argument("--batch-stride", type=int, default=1,
                    help="--batched-ops: every k-th instance of the draw (the draw is sorted by size)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="batched run: keep the default tile rule instead of the autotuner's choice")
    ap.add_argument("--learned", action="store_true",
                    help="the learned-iterate workload (2D 1025^2, 1000 fractures, trained U-Net)")
    ap.add_argument("--traj", type=int, default=200, help="--learned: training trajectories")
    ap.add_argument("--traj-steps", type=int, default=20, help="--learned: pressure steps per trajectory")
    ap.add_argument("--heldout", type=int, default=20, help="--learned: held-out trajectories")
    ap.add_argument("--fractures", type=int, default=1000, help="--learned: line fractures per network")
    ap.add_argument("--train-steps", type=int, default=2000, help="--learned: Adam steps (batch 4)")
    ap.add_argument("--traj-batch", type=int, default=8,
                    help="--learned: trajectories generated concurrently")
    ap.add_argument("--unet-kernels", action="store_true",
                    help="time the U-Net's tensor-core convolutions on a --unet-size grid")
    ap.add_argument("--unet-size", type=int, default=1032)
    ap.add_argument("--paper-scale", action="store_true",
                    help="the paper's 3D scenario at its size (393^3, 242.8M dofs, 100 plates)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched-ops", action="store_true",
                    help="skip the batched 2D product measurement of the default line")
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


def shard_instances(n, rank, world):
    """The instances of an n-instance batch that rank `rank` of `world`
    solves: round-robin, so every rank gets a like mix of the draw's sizes
    (the draw is sorted by size) and every instance is solved once."""
    return [i for i in range(n) if i % world == rank]


def batched_job(rank_seconds, rank_dofs, dist=None, device="cpu"):
    """Strong scaling of the batched workload over the ranks: each rank
    times its own share of the instances; the job lasts as long as the
    slowest rank and covers every rank's dofs.  Returns (the slowest rank's
    seconds per batch step, the batch's total dofs); a collective call."""
    if dist is None:
        return rank_seconds, rank_dofs
    import torch
    t = torch.tensor([float(rank_seconds)], dtype=torch.float64, device=device)
    d = torch.tensor([float(rank_dofs)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(d, op=dist.ReduceOp.SUM)
    return float(t.item()), int(d.item())


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
# The FP64 oracle (numpy) is timed in a child process of this script
# (`bench.py --oracle-worker SPEC`), so that its BLAS/OpenMP thread count can
# be fixed before numpy loads: once at one thread and once at the default
# (every core this process may use).  Nothing is scaled: each figure is the
# wall time of what ran.
THREAD_ENV = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS")


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count()


def cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        for line in open("/proc/cpuinfo"):
            low = line.lower()
            if low.startswith("model name") or low.startswith("cpu part") or low.startswith("hardware"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


def oracle_state(W):
    """The fractured initial state of workload W for the oracle."""
    from oracle import pf_oracle as O
    H = O.Hierarchy(3, W["n_coarse"], W["h_coarse"], W["levels"],
                    O.Params(E=W["E"], nu=W["nu"], Gc=W["Gc"], p=W["dp"]),
                    ls_over_h=W["ls_over_h"])
    g = H.fine
    x = np.zeros(4 * g.N)
    x[3 * g.N:] = O.rasterize(g, O.DISC3D, PI.disc_network_3d(W["seed"], W["fractures"]), g.h)
    return O, H, x


def oracle_worker(spec):
    """Runs inside the child process.  spec["kind"]:
    - "load_steps": run steps k = 1 .. warmup untimed and k = warmup+1 ..
      warmup+steps timed, each one whole oracle load step (Algorithm 1 V-cycles
      to the stopping test) at ramp pressure dp * ramp_t(k);
    - "passes": one hessvec, gradient and energy-difference pass each on the
      full finest state of the workload."""
    W = WORKLOAD_SMALL if spec["workload"] == "small" else WORKLOAD
    O, H, x0 = oracle_state(W)
    out = {"workload": W["workload"], "dofs": int(x0.size)}
    if spec["kind"] == "load_steps":
        x = x0.copy()
        secs, energies, cycles = [], [], []
        for k in range(1, spec["warmup"] + spec["steps"] + 1):
            t = ramp_t(k)
            if t == 1:
                x = x0.copy()
            t0 = time.perf_counter()
            r = O.rmtr_load_step(H, x, p=W["dp"] * t)
            dt = time.perf_counter() - t0
            x = r.x
            if k > spec["warmup"]:
                secs.append(dt)
                energies.append(r.energy)
                cycles.append(r.cycles)
        out.update(seconds=secs, energy=energies, cycles=cycles,
                   pressures=[W["dp"] * ramp_t(k) for k in
                              range(spec["warmup"] + 1, spec["warmup"] + spec["steps"] + 1)])
    else:
        g = H.fine
        x = x0.copy()
        x[:3 * g.N] = PI.random_direction(5, 3 * g.N, 1e-4)
        v = PI.random_direction(6, x.size, 1e-4)
        res = {}
        for name, fn in (("hessvec", lambda: O.hessvec(g, H.prm, x, v)),
                         ("gradient", lambda: O.gradient(g, H.prm, x)),
                         ("energy_diff", lambda: O.energy_diff(g, H.prm, x, v))):
            if name not in spec.get("passes", ("hessvec", "gradient", "energy_diff")):
                continue
            t0 = time.perf_counter()
            fn()
            dt = time.perf_counter() - t0
            res[name] = {"seconds": dt, "gdofs": x.size / dt / 1e9}
        out["passes"] = res
    print("ORACLE_RESULT " + json.dumps(out))
    return 0


def run_oracle(spec, threads=None, timeout=1500):
    """The oracle worker in a fresh child process; threads = 1 pins every
    BLAS/OpenMP pool to one thread, None leaves the defaults (all cores)."""
    env = dict(os.environ)
    for k in THREAD_ENV:
        env.pop(k, None)
        if threads is not None:
            env[k] = str(threads)
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-worker", json.dumps(spec)],
                       env=env, capture_output=True, text=True, timeout=timeout)
    for line in r.stdout.splitlines():
        if line.startswith("ORACLE_RESULT "):
            out = json.loads(line[len("ORACLE_RESULT "):])
            out["threads"] = threads if threads is not None else cpu_cores()
            return out
    raise RuntimeError(f"oracle worker failed (rc {r.returncode}): {r.stderr[-2000:]}")


def workload_config(W, args, world, **extra):
    """The workload a line reports: grid, sizes, the timed pressures and the
    solver settings."""
    n = [(c - 1) * (1 << (W["levels"] - 1)) + 1 for c in W["n_coarse"]]
    cfg = {"workload": W["workload"], "grid": n, "levels": W["levels"],
           "dofs": (W["dim"] + 1) * int(np.prod(n)), "fractures": W["fractures"],
           "ramp": f"p_t = {W['dp']} t, t = 1..{RAMP}; run step k solves t = (k-1) mod {RAMP} + 1, "
                   "restarting from the fractured state at t = 1",
           "pressure_steps": [W["dp"] * ramp_t(k)
                              for k in range(args.warmup + 1, args.warmup + args.steps + 1)],
           "parallelism": f"replicas{world}",
           "l2": "working set > L2 (FP64 vectors 69 MB each, >20 resident)"}
    cfg.update(extra)
    return cfg


def run_reference(args):
    """The reference arm: the FP64 oracle (the paper ships no code), run as it
    stands on this machine's host cores.  A whole oracle load step of the
    129^3 workload takes hours, so every step here is one whole oracle load
    step of the same workload eight times coarser per axis (17^3, four
    levels, the same discs, material and ramp), timed as it ran."""
    rank, world, _ = rank_info()
    if rank != 0:
        return 0
    W = WORKLOAD_SMALL
    allc = run_oracle({"kind": "load_steps", "workload": "small", "warmup": args.warmup,
                       "steps": args.steps})
    one = run_oracle({"kind": "load_steps", "workload": "small", "warmup": 0, "steps": 2}, threads=1)
    passes = run_oracle({"kind": "passes", "workload": "full"})
    v = sum(allc["seconds"]) / args.steps
    out = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": v * 1e3,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": workload_config(W, args, world, precision="fp64", start="plain",
                                  coarse_model="first_order", solver="FP64 numpy oracle",
                                  l2="host CPU run (no GPU)"),
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": allc["threads"], "kind": "oracle",
                         "cpu": cpu_model(), "nproc": os.cpu_count(),
                         "sample": (f"{args.steps} whole oracle load steps (after {args.warmup} untimed) of "
                                    f"{W['workload']} ({allc['dofs']} dofs), default BLAS threads; "
                                    "nothing scaled"),
                         "seconds": allc["seconds"], "cycles": allc["cycles"],
                         "one_thread": {"seconds": one["seconds"], "pressures": one["pressures"],
                                        "value": sum(one["seconds"]) / len(one["seconds"])},
                         "passes_129": {"threads": passes["threads"], **passes["passes"]}},
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


def undetermined_nodes(c, n):
    """Nodes whose every element has c = 1 at all eight corners: g(c) = 0 at
    every Gauss point around them, so their displacements carry no energy
    and any value minimises (such dofs are left out of field comparisons)."""
    import torch
    full = (c.view(n[2], n[1], n[0]) == 1.0)
    e = torch.ones(n[2] + 1, n[1] + 1, n[0] + 1, dtype=torch.bool, device=c.device)
    inner = full[:-1, :-1, :-1].clone()
    for dz in (0, 1):
        for dy in (0, 1):
            for dx in (0, 1):
                inner &= full[dz:dz + n[2] - 1, dy:dy + n[1] - 1, dx:dx + n[0] - 1]
    e[1:-1, 1:-1, 1:-1] = inner
    und = torch.ones(n[2], n[1], n[0], dtype=torch.bool, device=c.device)
    for dz in (0, 1):
        for dy in (0, 1):
            for dx in (0, 1):
                und &= e[dz:dz + n[2], dy:dy + n[1], dx:dx + n[0]]
    return und.reshape(-1)


def field_errors(xm, xf, n):
    """Per-field error of the state xm against the FP64 state xf: the largest
    absolute difference, that over the field's max-norm, and the relative L2
    error, on every determined dof (undetermined displacements excluded)."""
    N = int(np.prod(n))
    und = undetermined_nodes(xf[3 * N:], n)
    out = {"undetermined_nodes": int(und.sum())}
    for f, name in enumerate(("u_x", "u_y", "u_z", "c")):
        a, b = xm[f * N:(f + 1) * N], xf[f * N:(f + 1) * N]
        d = (a - b)
        if f < 3:
            d = d.masked_fill(und, 0.0)
            b = b.masked_fill(und, 0.0)
        bmax = float(b.abs().max())
        dmax = float(d.abs().max())
        out[name] = {"max_abs": dmax, "max_rel": dmax / bmax if bmax > 0 else dmax,
                     "rel_l2": float(d.norm()) / max(float(b.norm()), 1e-300)}
    return out


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
    prec = pf.PF_FP32 if args.precision == "mixed" else pf.PF_FP64
    cmodel = pf.PF_GALERKIN if args.coarse_model == "galerkin" else pf.PF_FIRST_ORDER
    start = pf.PF_START_EXTRAPOLATE if args.start == "extrapolate" else pf.PF_START_PLAIN

    def make(Wx):
        Hx = pf.mesh_hierarchy_create(3, Wx["n_coarse"], Wx["levels"], Wx["h_coarse"], E=Wx["E"],
                                      nu=Wx["nu"], Gc=Wx["Gc"], ls_over_h=Wx["ls_over_h"])
        xx = torch.zeros(Hx.ndof(), dtype=torch.float64, device="cuda")
        pf.fractures_set(Hx, pf.PF_DISC3D, PI.disc_network_3d(Wx["seed"], Wx["fractures"]),
                         Hx.levels[-1][1], xx)
        return Hx, xx

    H, x = make(W)
    g_n, g_h, N = H.levels[-1]
    ndof = H.ndof()
    x_frac = x.clone()  # the fractured initial state every ramp starts from
    stream = torch.cuda.current_stream()

    if args.kernels_only:
        return kernels_only(pf, B, H, x, W)

    def params(precision, st, t, dp, model=None):
        """Parameters of ramp step t: the previous ramp pressure names the
        extrapolation's base, so every arm extrapolates alike."""
        return pf.default_params(precision=precision, coarse_model=cmodel if model is None else model,
                                 start=st, p_prev=dp * (t - 1) if t > 1 else 0.0)

    def load_step(Hx, xx, xfrac, k, precision, st, dp, model=None):
        t = ramp_t(k)
        if t == 1:
            xx.copy_(xfrac)
        pf.pressure_set(Hx, dp * t)
        return pf.rmtr_load_step(Hx, xx, params(precision, st, t, dp, model), check=False)

    first, last = args.warmup + 1, args.warmup + args.steps
    for k in range(1, args.warmup + 1):
        load_step(H, x, x_frac, k, prec, start, W["dp"])
    x_after_warmup = x.clone()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = Clocks(local)
    clocks.start()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    stats = []
    ev[0].record(stream)
    with nvtx_range("timed_load_steps"):  # ncu --nvtx-include "timed_load_steps/"
        for j, k in enumerate(range(first, last + 1)):
            stats.append(load_step(H, x, x_frac, k, prec, start, W["dp"]))
            ev[j + 1].record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    step_s = [ev[j].elapsed_time(ev[j + 1]) * 1e-3 for j in range(args.steps)]
    slowest_s, job_s = job_seconds_per_load_step(ev[0].elapsed_time(ev[-1]) / args.steps / 1e3,
                                                 dist, "cuda")
    ms = slowest_s * 1e3
    if dist:
        dist.barrier()

    # ---- dominant kernel: Hessian-vector product at the finest level.
    # Launches rotate over four independent operand sets (together well
    # above L2), so no launch finds its inputs in L2.
    level = W["levels"] - 1
    vs = [torch.from_numpy(PI.random_direction(77 + i, ndof, 1e-3)).cuda() for i in range(4)]
    outs = [torch.empty_like(vs[0]) for _ in range(4)]
    xs32 = [(x + 1e-6 * vs[(i + 1) % 4]).float() for i in range(4)]
    vs32 = [v.float() for v in vs]
    os32 = [torch.empty_like(vs32[0]) for _ in range(4)]

    def time_kernel(fn, reps=20):
        for i in range(4):
            fn(i)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for r in range(reps):
            fn(r % 4)
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps * 1e-3

    pf.hessvec_lag_set(H, level, x)  # the solver's FP64 operator: stored lagged coefficients
    kclocks = Clocks(local)
    kclocks.start()
    t64 = time_kernel(lambda i: pf.hessvec_lagged(H, level, vs[i], outs[i]))
    t32 = time_kernel(lambda i: pf.hessvec(H, level, xs32[i], vs32[i], os32[i]), reps=40)
    t_grad = time_kernel(lambda i: pf.gradient(H, level, x, outs[i]))
    kclk = kclocks.stop()
    fma64 = B.probe_fma(pf.PF_FP64)
    fma32 = B.probe_fma(pf.PF_FP32)
    try:
        hbm = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"]
        hbm_src = "measured"
    except (OSError, KeyError, ValueError):
        hbm, hbm_src = 6800.0, "fallback"
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    sm_mhz = kclk["sm_mhz"] or clk["sm_mhz"] or 2070.0
    fp32_peak = sms * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12
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
    # The FP32 product is bound by FP32 issue: ALU roofline, algorithmic
    # flops = FLOP32_PER_ELEMENT x elements
    ne = (g_n[0] - 1) * (g_n[1] - 1) * (g_n[2] - 1)
    flops32 = FLOP32_PER_ELEMENT * ne
    roof32 = {"kernel": "hessvec_fp32", "bound": "alu", "achieved": flops32 / t32 / 1e12,
              "peak": fp32_peak, "unit": "TFLOP/s",
              "frac": flops32 / t32 / 1e12 / fp32_peak,
              # dram__bytes_read.sum + dram__bytes_write.sum of one ncu capture of
              # the product's two kernels
              "traffic": TRAFFIC_HESSVEC_FP32,
              "peak_source": (f"derived: {sms} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 flop x "
                              f"{sm_mhz:.0f} MHz (median SM clock sampled while the kernels ran)"),
              "fp32_fma_probe_tflops": fma32 / 1e12,
              "flop_per_element": FLOP32_PER_ELEMENT,
              "hbm_achieved_gbs": bytes32 / t32 / 1e9, "hbm_peak_gbs": hbm,
              "hbm_frac": bytes32 / t32 / 1e9 / hbm,
              "gdofs": ndof / t32 / 1e9, "us_per_launch": t32 * 1e6,
              "operands": "4 rotating operand sets (x_lag, v, Hv), 412 MB, above L2"}
    roofline = roof64 if args.precision == "fp64" else roof32

    # ---- the metric's comparison: the same ramp steps from the same warmed
    # state in plain FP64 (plain start) and in mixed precision with the plain
    # start, beside a re-run of the headline's own steps (bitwise the same
    # solves: the solver is deterministic) whose states give the per-field
    # error of the mixed fields against the FP64 fields at every step.
    cmp = None
    if not args.no_compare:
        n_cmp = min(args.steps, RAMP)
        ks = list(range(first, first + n_cmp))

        def arm(precision, st, keep=False, model=None):
            xx = x_after_warmup.clone()
            torch.cuda.synchronize()
            secs, sts, states = [], [], []
            for k in ks:
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record(stream)
                sts.append(load_step(H, xx, x_frac, k, precision, st, W["dp"], model))
                b.record(stream)
                torch.cuda.synchronize()
                secs.append(a.elapsed_time(b) * 1e-3)
                if keep:
                    states.append(xx.clone())
            return secs, sts, states, xx

        m_s, m_st, m_states, _ = arm(prec, start, keep=True)
        f_s, f_st, f_states, _ = arm(pf.PF_FP64, pf.PF_START_PLAIN, keep=True)
        p_s, p_st, _, _ = arm(pf.PF_FP32, pf.PF_START_PLAIN)
        # the paper's second-order coarse model (stored FP32 Galerkin
        # operators) beside the first-order one, headline settings otherwise
        other = pf.PF_FIRST_ORDER if cmodel == pf.PF_GALERKIN else pf.PF_GALERKIN
        o_s, o_st, _, _ = arm(prec, start, model=other)
        errs = [field_errors(a, b, g_n) for a, b in zip(m_states, f_states)]
        del m_states, f_states
        worst = {f: {m: max(e[f][m] for e in errs) for m in ("max_abs", "max_rel", "rel_l2")}
                 for f in ("u_x", "u_y", "u_z", "c")}
        mixed_mean = sum(m_s) / n_cmp
        fp64_mean = sum(f_s) / n_cmp
        cmp = {
            "steps": ks, "pressures": [W["dp"] * ramp_t(k) for k in ks],
            "fp64_plain": {"value": fp64_mean, "unit": UNIT, "seconds": f_s,
                           "cycles": [s["cycles"] for s in f_st], "status": [s["status"] for s in f_st],
                           "energy": [s["energy"] for s in f_st]},
            "mixed_plain_start": {"value": sum(p_s) / n_cmp, "unit": UNIT, "seconds": p_s,
                                  "cycles": [s["cycles"] for s in p_st]},
            "headline_same_steps": {"value": mixed_mean, "unit": UNIT, "seconds": m_s,
                                    "cycles": [s["cycles"] for s in m_st],
                                    "bitwise_as_timed": all(a["energy"] == b["energy"]
                                                            for a, b in zip(m_st, stats))},
            "other_coarse_model": {"coarse_model": "galerkin" if other == pf.PF_GALERKIN else "first_order",
                                   "value": sum(o_s) / n_cmp, "unit": UNIT, "seconds": o_s,
                                   "cycles": [s["cycles"] for s in o_st],
                                   "energy_rel_diff": max(abs(a["energy"] - b["energy"]) / abs(b["energy"])
                                                          for a, b in zip(o_st, f_st))},
            "fp64_plain_over_headline": fp64_mean / mixed_mean,
            "energy_rel_diff": max(abs(a["energy"] - b["energy"]) / abs(b["energy"])
                                   for a, b in zip(m_st, f_st)),
            "field_error_vs_fp64": {"per_step": errs, "worst": worst},
        }

    # ---- end to end through the host-buffer entry point
    e2e = None
    if not args.no_e2e:
        xh = torch.empty(ndof, dtype=torch.float64, pin_memory=True)
        xh.copy_(x_after_warmup.cpu())
        xfh = x_frac.cpu().numpy()
        xn = xh.numpy()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k in range(first, last + 1):
            t = ramp_t(k)
            if t == 1:
                xn[:] = xfh
            pf.pressure_set(H, W["dp"] * t)
            pf.rmtr_load_step_host(H, xn, params(prec, start, t, W["dp"]), check=False)
        _, e2e_s = job_seconds_per_load_step((time.perf_counter() - t0) / args.steps, dist, "cuda")
        e2e = {"value": e2e_s, "unit": UNIT, "h2d_bytes_per_step": 8 * ndof,
               "d2h_bytes_per_step": 8 * ndof}

    # ---- the FP64 oracle on this machine's host cores (rank 0 at N = 1):
    # whole oracle load steps of the 17^3 workload and one pass each at
    # 129^3, timed as they ran, beside the GPU on the same 17^3 steps
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        n_s = 3
        allc = run_oracle({"kind": "load_steps", "workload": "small", "warmup": 0, "steps": n_s})
        one = run_oracle({"kind": "load_steps", "workload": "small", "warmup": 0, "steps": 1},
                         threads=1)
        pass_all = run_oracle({"kind": "passes", "workload": "full"})
        pass_one = run_oracle({"kind": "passes", "workload": "full", "passes": ["hessvec"]},
                              threads=1)
        Hs, xs_ = make(WORKLOAD_SMALL)
        xs_frac = xs_.clone()
        gpu_small = {}
        for name, pr, st in (("headline", prec, start), ("fp64_plain", pf.PF_FP64, pf.PF_START_PLAIN)):
            for k in range(1, n_s + 1):  # warm-up: graphs and lag buffers of this hierarchy
                load_step(Hs, xs_, xs_frac, k, pr, st, WORKLOAD_SMALL["dp"])
            secs, en = [], []
            for k in range(1, n_s + 1):
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record(stream)
                s_ = load_step(Hs, xs_, xs_frac, k, pr, st, WORKLOAD_SMALL["dp"])
                b.record(stream)
                torch.cuda.synchronize()
                secs.append(a.elapsed_time(b) * 1e-3)
                en.append(s_["energy"])
            gpu_small[name] = {"seconds": secs, "value": sum(secs) / n_s, "energy": en}
        Hs.close()
        v_or = sum(allc["seconds"]) / n_s
        cpu = {"value": v_or, "unit": UNIT, "cores": allc["threads"], "kind": "oracle",
               "cpu": cpu_model(), "nproc": os.cpu_count(),
               "sample": (f"whole FP64 oracle load steps t = 1..{n_s} of {WORKLOAD_SMALL['workload']} "
                          f"({allc['dofs']} dofs: the timed workload eight times coarser per axis), "
                          "default BLAS threads, timed as they ran (nothing scaled); plus one "
                          "hessvec / gradient / energy-difference pass on the full 129^3 state"),
               "seconds": allc["seconds"], "cycles": allc["cycles"],
               "one_thread": {"seconds": one["seconds"], "value": one["seconds"][0]},
               "passes_129": {"all_cores": {"threads": pass_all["threads"], **pass_all["passes"]},
                              "one_thread": pass_one["passes"]},
               "equal_work_17": {
                   "workload": WORKLOAD_SMALL["workload"], "pressures": allc["pressures"],
                   "oracle": v_or, "gpu_headline": gpu_small["headline"]["value"],
                   "gpu_fp64_plain": gpu_small["fp64_plain"]["value"],
                   "oracle_over_gpu_headline": v_or / gpu_small["headline"]["value"],
                   "oracle_over_gpu_fp64_plain": v_or / gpu_small["fp64_plain"]["value"],
                   "fp64_energy_rel_diff_vs_oracle": max(
                       abs(a - b) / abs(b) for a, b in zip(gpu_small["fp64_plain"]["energy"],
                                                            allc["energy"])),
                   "headline_energy_rel_diff_vs_oracle": max(
                       abs(a - b) / abs(b) for a, b in zip(gpu_small["headline"]["energy"],
                                                            allc["energy"]))},
               "hessvec_129_gpu_fp32_over_oracle": (pass_all["passes"]["hessvec"]["seconds"] / t32)}

    # ---- the batched workload's data-parallel kernel: the FP32 Hessian
    # product of the 64 uneven 2D instances in one persistent launch
    bops = None
    if rank == 0 and world == 1 and not args.no_batched_ops:
        _, _, Hb, xb = batched_instances(pf, torch, 64, True)
        for Hh in Hb:
            pf.pressure_set(Hh, 1e-3)
        bclk = Clocks(0)
        bclk.start()
        bops = time_batched_ops(pf, torch, Hb, xb, 20)
        bops["clocks"] = bclk.stop()
        for Hh in Hb:
            Hh.close()
        del Hb, xb
        torch.cuda.empty_cache()

    launches = int(sum(s["launches"] for s in stats))
    value = job_s
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if args.precision == "fp64" else "f64+f32",
            "data": "synthetic",
            "config": workload_config(
                W, args, world, precision=args.precision, coarse_model=args.coarse_model,
                start=args.start if args.start == "plain" else
                "extrapolate (the learned iterate's zero-output predictor; the network is 2D)"),
            "seconds_per_step": step_s,
            "roofline": roofline,
            "roofline_other": roof32 if roofline is roof64 else roof64,
            "hessvec_gdofs": {"fp64": ndof / t64 / 1e9, "fp32": ndof / t32 / 1e9},
            "gradient_fp64_us": t_grad * 1e6,
            "fp64_plain": cmp["fp64_plain"] if cmp else None,
            "compare": cmp,
            "clocks": clk,
            "kernel_clocks": kclk,
            "e2e": e2e,
            "gpu_launches": launches,
            "cpu_baseline": cpu,
            "batched_hessvec": bops,
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


def run_paper_scale(args):
    """Load steps of the paper's 242.8M-dof 3D scenario on one GPU (mixed
    precision, extrapolated start): W untimed steps k = 0 .. W-1, then K
    timed steps, each timed with CUDA events; plus the FP32 Hessian
    product's time at this size."""
    import torch
    from paper_2007_12908_gb300 import build
    build.build()
    import paper_2007_12908_gb300 as pf
    W = PAPER_SCALE
    H = pf.mesh_hierarchy_create(3, W["n_coarse"], W["levels"], W["h_coarse"], E=W["E"], nu=W["nu"],
                                 Gc=W["Gc"], ls_over_h=W["ls_over_h"])
    x = torch.zeros(H.ndof(), dtype=torch.float64, device="cuda")
    g_n, g_h, N = H.levels[-1]
    pf.fractures_set(H, pf.PF_BOX3D, PI.box_network_3d(W["seed"], W["fractures"]), g_h, x)
    stream = torch.cuda.current_stream()
    prec = pf.PF_FP32 if args.precision == "mixed" else pf.PF_FP64

    def step(k):
        p = W["p0"] + k * W["dp"]
        pf.pressure_set(H, p)
        prm = pf.default_params(precision=prec, start=pf.PF_START_EXTRAPOLATE,
                                p_prev=(W["p0"] + (k - 1) * W["dp"]) if k > 0 else 0.0)
        return pf.rmtr_load_step(H, x, prm, check=False)

    for k in range(args.warmup):
        step(k)
    torch.cuda.synchronize()
    clocks = Clocks(0)
    clocks.start()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    stats = []
    ev[0].record(stream)
    for j, k in enumerate(range(args.warmup, args.warmup + args.steps)):
        stats.append(step(k))
        ev[j + 1].record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    secs = [ev[j].elapsed_time(ev[j + 1]) * 1e-3 for j in range(args.steps)]
    level = W["levels"] - 1
    ndof = H.ndof()
    v32 = torch.from_numpy(PI.random_direction(78, ndof, 1e-3)).cuda().float()
    x32, o32 = x.float(), torch.empty_like(v32)
    for _ in range(3):
        pf.hessvec(H, level, x32, v32, o32)
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(10):
        pf.hessvec(H, level, x32, v32, o32)
    b.record(stream)
    torch.cuda.synchronize()
    t32 = a.elapsed_time(b) / 10 * 1e-3
    ne = (g_n[0] - 1) * (g_n[1] - 1) * (g_n[2] - 1)
    free_b, total_b = torch.cuda.mem_get_info()
    line = {
        "metric": "RMTR s/load-step at the paper's 3D size", "value": sum(secs) / args.steps,
        "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "higher_is_better": False, "dtype": "f64+f32" if prec == pf.PF_FP32 else "f64",
        "data": "synthetic",
        "config": {"workload": W["workload"], "grid": list(g_n), "levels": W["levels"], "dofs": ndof,
                   "fractures": W["fractures"], "E": W["E"], "nu": W["nu"], "Gc": W["Gc"],
                   "pressures": [W["p0"] + k * W["dp"] for k in range(args.warmup, args.warmup + args.steps)],
                   "precision": args.precision, "start": "extrapolate"},
        "seconds_per_step": secs,
        "solver": {k: [s_[k] for s_ in stats] for k in ("cycles", "converged", "cg", "status", "energy")},
        "hessvec_fp32": {"us_per_launch": t32 * 1e6, "gdofs": ndof / t32 / 1e9,
                         "tflops": FLOP32_PER_ELEMENT * ne / t32 / 1e12},
        "device_memory_used_gb": (total_b - free_b) / 1e9,
        "clocks": clk,
    }
    print(json.dumps(line))
    H.close()
    return 0


def run_learned(args):
    """The learned-initial-iterate workload: 2D 1025^2 grid (seven levels from
    17^2), 1,000 line fractures per trajectory, the ramp p_t = 5e-4 t,
    t = 1..20.  Trains the U-Net on args.traj solver trajectories (each its own
    seeded network) with the library's forward/backward/Adam kernels, then
    runs args.heldout held-out trajectories from the plain, the extrapolated
    and the learned start, reporting V-cycles and seconds per load step."""
    import torch
    from paper_2007_12908_gb300 import build
    build.build()
    import paper_2007_12908_gb300 as pf
    from paper_2007_12908_gb300 import learned as Lm
    steps = args.traj_steps
    pressures = [5e-4 * t for t in range(1, steps + 1)]
    H = pf.mesh_hierarchy_create(2, (17, 17), 7, 1 / 16, E=1.0, nu=0.3, Gc=1.0)
    (nx, ny), h, N = H.levels[-1]
    # the solver settings of this workload: the crack networks converge
    # slowly with first-order coarse models (50-80+ V-cycles per step), so the
    # stored Galerkin operators with 50 CG iterations per coarse smoothing
    # step and 200 on the finest level
    solver = dict(precision=pf.PF_FP32, coarse_model=pf.PF_GALERKIN, cg_smooth=50, cg_fine=200)
    prm = pf.default_params(start=pf.PF_START_EXTRAPOLATE, **solver)

    def network(seed, Hh=None):
        """The seeded network's fractures in x0 and in Hh's c_prev (the
        irreversibility bound belongs to the hierarchy that solves it)."""
        Hh = H if Hh is None else Hh
        x0 = torch.zeros(H.ndof(), dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        pf.fractures_set(Hh, pf.PF_LINE2D, PI.line_network_2d(seed, args.fractures), h, x0)
        torch.cuda.synchronize()
        return x0

    learner = Lm.LearnedIterate(H, seed=1)
    data = []
    t0 = time.perf_counter()
    # trajectories in groups of --traj-batch, each group's load steps run
    # concurrently on hierarchies of their own (one stream each)
    K = max(1, args.traj_batch)
    Hg = [H] + [pf.mesh_hierarchy_create(2, (17, 17), 7, 1 / 16, E=1.0, nu=0.3, Gc=1.0,
                                         stream=torch.cuda.Stream()) for _ in range(K - 1)]
    for k0 in range(0, args.traj, K):
        ks = list(range(k0, min(args.traj, k0 + K)))
        x0s = [network(PI.SEED_2D_LEARNED + k, Hg[j]) for j, k in enumerate(ks)]
        if K == 1:
            group = [Lm.trajectory(H, x0s[0], pressures, prm)]
        else:
            group = Lm.trajectories(Hg[:len(ks)], x0s, pressures, prm)
        for states in group:
            data += Lm.samples(learner, states, pressures)
        del group, x0s
        print(f"trajectories {ks[-1] + 1}/{args.traj}: {len(data)} samples, {time.perf_counter() - t0:.0f} s",
              file=sys.stderr, flush=True)
    for Hh in Hg[1:]:
        Hh.close()
    t_data = time.perf_counter() - t0
    t1 = time.perf_counter()
    losses = Lm.train(learner, data, steps=args.train_steps, lr=1e-3, batch=4)
    t_train = time.perf_counter() - t1
    del data
    torch.cuda.empty_cache()
    res = {m: [] for m in ("plain", "extrapolated", "learned")}
    plain_prm = pf.default_params(**solver)
    for k in range(args.heldout):
        x0 = network(PI.SEED_2D_LEARNED + 100000 + k)
        for mode in res:
            recs, _ = Lm.run_ramp(H, x0, pressures, plain_prm, mode=mode, learner=learner)
            res[mode].append(recs)
        print(f"held-out {k + 1}/{args.heldout}", file=sys.stderr, flush=True)
    summary = {}
    for mode, runs in res.items():
        later = [r for recs in runs for r in recs[1:]]
        summary[mode] = {"v_cycles_per_step": statistics.mean(r["cycles"] for r in later),
                         "s_per_load_step": statistics.mean(r["seconds"] for r in later),
                         "converged": all(r["converged"] for recs in runs for r in recs)}
    acc = [r.get("accepted", False) for recs in res["learned"] for r in recs[1:]]
    acc_e = [r.get("accepted_extrapolated", False) for recs in res["learned"] for r in recs[1:]]
    line = {
        "metric": "learned initial iterate: V-cycles and s/load-step (t >= 2) on held-out trajectories",
        "value": summary["learned"]["s_per_load_step"], "unit": UNIT, "higher_is_better": False,
        "n_gpus": 1, "data": "synthetic",
        "config": {"workload": "2d_1025^2_q1_7level_1000lines_ramp20", "grid": [nx, ny], "levels": 7,
                   "dofs": H.ndof(), "fractures": args.fractures, "pressure_steps": pressures,
                   "training_trajectories": args.traj, "heldout_trajectories": args.heldout,
                   "trajectories_generated_concurrently": max(1, args.traj_batch),
                   "samples": args.traj * (steps - 1), "adam_steps": args.train_steps, "batch": 4,
                   "precision": "mixed", "coarse_model": "galerkin", "cg_smooth": 50, "cg_fine": 200,
                   "network": "U-Net 16-32-64-128, BF16, tensor-core convolutions"},
        "starts": summary,
        "gain_v_cycles": {"over_plain": summary["plain"]["v_cycles_per_step"] - summary["learned"]["v_cycles_per_step"],
                          "over_extrapolated": summary["extrapolated"]["v_cycles_per_step"]
                          - summary["learned"]["v_cycles_per_step"]},
        "gate_accepted": {"network": statistics.mean(1.0 if a else 0.0 for a in acc),
                          "extrapolation": statistics.mean(1.0 if a else 0.0 for a in acc_e)},
        "loss": {"first": float(np.mean(losses[:10])), "last": float(np.mean(losses[-10:]))},
        "seconds": {"trajectories": t_data, "training": t_train},
    }
    print(json.dumps(line))
    H.close()
    return 0


def run_unet_kernels(args):
    """The learned iterate's U-Net on an S x S grid (the 1025^2 workload pads
    to 1032): forward and backward times of the tensor-core convolution
    kernels and their rate against the measured BF16 peak."""
    import torch
    from paper_2007_12908_gb300 import build
    build.build()
    from paper_2007_12908_gb300 import _binding as B
    from paper_2007_12908_gb300 import learned as Lm
    S = args.unet_size
    net = B.Unet(S, S)
    net.set_params(Lm.he_init(3))
    g = torch.Generator(device="cuda")
    g.manual_seed(5)
    x = torch.randn(5, S, S, device="cuda", generator=g)
    t = torch.randn(3, S, S, device="cuda", generator=g)
    flops = 0
    shapes = Lm.layer_shapes()
    lev = [0, 0, 1, 1, 2, 2, 3, 3, 2, 2, 1, 1, 0, 0, 0]
    for (co, ci, k), l in zip(shapes, lev):
        flops += 2 * (S >> l) * (S >> l) * co * ci * k * k
    for _ in range(3):
        y = net.forward(x)
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(args.steps):
        y = net.forward(x)
    b.record()
    torch.cuda.synchronize()
    t_f = a.elapsed_time(b) / args.steps * 1e-3
    _, dy = net.mse(y, t)
    net.backward(dy)
    torch.cuda.synchronize()
    a.record()
    for _ in range(args.steps):
        net.backward(dy)
    b.record()
    torch.cuda.synchronize()
    t_b = a.elapsed_time(b) / args.steps * 1e-3
    try:
        peak = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["bf16_tflops_sustained"]
        src = "measured (MEASURED_PEAKS.json bf16_tflops_sustained)"
    except (OSError, KeyError, ValueError):
        peak, src = 1700.0, "fallback"
    print(json.dumps({"unet": {"grid": S, "flop_forward": flops, "forward_ms": t_f * 1e3,
                               "forward_tflops": flops / t_f / 1e12, "backward_ms": t_b * 1e3,
                               "backward_tflops": 2 * flops / t_b / 1e12,
                               "forward_frac": flops / t_f / 1e12 / peak, "peak_tflops": peak,
                               "peak_source": src}}))
    return 0


def time_batched_ops(pf, torch, Hs, states, K, bps=0):
    """The batched FP32 Hessian product over every instance in one persistent
    launch (pf_batch_hessvec): microseconds per launch with CUDA events on
    the batch's stream, HBM rate at the algorithmic 12 B/dof (x, v read, Hv
    written; the vectors exceed L2), against the same products launched
    one instance at a time."""
    st = torch.cuda.Stream()
    g = torch.Generator(device="cuda")
    g.manual_seed(17)
    xs, vs, ys = [], [], []
    for H, x in zip(Hs, states):
        N = H.nodes()
        x32 = x.float()
        x32[:2 * N] += 1e-3 * torch.randn(2 * N, device="cuda", generator=g)
        xs.append(x32)
        vs.append(torch.randn(3 * N, device="cuda", generator=g))
        ys.append(torch.empty(3 * N, device="cuda"))
    torch.cuda.synchronize()
    with torch.cuda.stream(st):
        B = pf.Batch(Hs, stream=st)
        if bps:  # a fixed launch configuration (e.g. under a profiler, whose replays skew the timings)
            B.variant_set(bps)
            tune_us = None
        else:
            bps, tune_us = B.autotune(xs, vs, ys)
        vhv = torch.empty(len(Hs), dtype=torch.float64, device="cuda")
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)

        def timed(dot):
            for _ in range(3):
                B.hessvec(xs, vs, ys, vhv=vhv if dot else None)
            a.record(st)
            for _ in range(K):
                B.hessvec(xs, vs, ys, vhv=vhv if dot else None)
            b.record(st)
            b.synchronize()
            return a.elapsed_time(b) * 1e3 / K

        us = timed(False)
        us_dot = timed(True)
    one = 0.0
    for H, x32, v, y in zip(Hs, xs, vs, ys):
        s2 = H.stream
        with torch.cuda.stream(s2):
            pf.hessvec(H, H.n_levels - 1, x32, v, out=y)
            a.record(s2)
            for _ in range(K):
                pf.hessvec(H, H.n_levels - 1, x32, v, out=y)
            b.record(s2)
        b.synchronize()
        one += a.elapsed_time(b) * 1e3 / K
    B.close()
    dofs = sum(H.ndof() for H in Hs)
    try:
        hbm = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"]
        src = "measured (MEASURED_PEAKS.json hbm_gbs)"
    except (OSError, KeyError, ValueError):
        hbm, src = 6800.0, "fallback"
    gbs = 12.0 * dofs / (us * 1e-6) / 1e9
    return {"kernel": "k_batch_hess2", "instances": len(Hs), "dofs": dofs, "us_per_launch": us,
            "us_per_launch_with_vHv": us_dot, "gdofs": dofs / us / 1e3, "achieved_gbs": gbs,
            "algorithmic_bytes": 12 * dofs, "peak_gbs": hbm, "hbm_frac": gbs / hbm, "peak_source": src,
            "blocks_per_sm": bps, "autotune_us": tune_us, "one_launch_per_instance_us": one,
            "speedup_vs_one_launch_per_instance": one / us, "launches_timed": K}


def batched_instances(pf, torch, count, streams, stride=1, pick=None):
    sizes, counts = PI.batched_grid_draw(PI.SEED_2D_BATCHED, 64)
    if pick is None:
        pick = list(range(0, 64, stride))[:count]
    Hs, xs = [], []
    for i in pick:
        n, nf = sizes[i], counts[i]
        levels = int(round(np.log2((n - 1) / 16))) + 1
        st = torch.cuda.Stream() if streams else None
        H = pf.mesh_hierarchy_create(2, (17, 17), levels, 1 / 16, E=1.0, nu=0.3, Gc=1.0, stream=st)
        x = torch.zeros(H.ndof(), dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        pf.fractures_set(H, pf.PF_LINE2D, PI.line_network_2d(PI.SEED_2D_BATCHED + 1 + i, nf),
                         H.levels[-1][1], x)
        Hs.append(H)
        xs.append(x)
    return [sizes[i] for i in pick], [counts[i] for i in pick], Hs, xs


def run_batched_ops(args):
    """Only the batched operators on the first --batch-count instances of the
    uneven 2D draw (all 64 by default)."""
    import torch
    from paper_2007_12908_gb300 import build
    build.build()
    import paper_2007_12908_gb300 as pf
    sizes, counts, Hs, xs = batched_instances(pf, torch, args.batch_count, True, args.batch_stride)
    for H in Hs:
        pf.pressure_set(H, 1e-3)
    clocks = Clocks(0)
    clocks.start()
    r = time_batched_ops(pf, torch, Hs, xs, args.steps, args.batch_bps)
    r["clocks"] = clocks.stop()
    r["sizes"] = sizes
    print(json.dumps({"batched_hessvec": r}))
    return 0


def run_batched(args):
    """Load steps of 64 uneven 2D instances (16 each of 129^2, 257^2, 513^2,
    1025^2 nodes; 10-1000 line fractures, +-30 deg families) run
    concurrently, each on its own stream, by the library's host workers."""
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
    prm = pf.default_params(precision=pf.PF_FP32 if args.precision == "mixed" else pf.PF_FP64,
                            start=pf.PF_START_EXTRAPOLATE if args.start == "extrapolate" else pf.PF_START_PLAIN)
    # the 64 instances are independent: each rank solves its share, no
    # collective on the data path
    sizes, counts, Hs, xs = batched_instances(pf, torch, 64, True, pick=shard_instances(64, rank, world))
    dofs = sum(H.ndof() for H in Hs)
    # the tile autotuner on every instance (per level: the fastest FP32
    # Hessian tile variant, measured), unless --no-autotune
    tuned = {}
    if not args.no_autotune:
        for H, n in zip(Hs, sizes):
            var, us = pf.autotune(H)
            tuned.setdefault(str(n), []).append(var)
        torch.cuda.synchronize()

    def step(t, threads):
        for H in Hs:
            pf.pressure_set(H, 1e-3 * t)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        t0 = time.perf_counter()
        out = pf.rmtr_load_step_batch(Hs, xs, prm, n_threads=threads, check=False)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
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
    sec, total_dofs = batched_job(statistics.mean(times), dofs, dist, "cuda")
    ops = time_batched_ops(pf, torch, Hs, xs, 20) if world == 1 else None
    if dist:
        dist.destroy_process_group()
    if rank != 0:
        return 0
    line = {
        "metric": "batched RMTR load steps: GDoF/s over 64 uneven 2D instances",
        "value": total_dofs / sec / 1e9, "unit": "GDoF/s (load steps)", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": sec * 1e3,
        "higher_is_better": True, "scaling": "strong", "vs_baseline": None,
        "dtype": "f64" if args.precision == "fp64" else "f64+f32", "data": "synthetic",
        "config": {"workload": "2d_batched_64_uneven_129-1025", "instances": 64, "dofs": total_dofs,
                   "instances_on_rank0": len(Hs), "sizes_on_rank0": sizes,
                   "fractures_on_rank0": counts, "precision": args.precision,
                   "start": args.start, "threads": args.batch_threads or len(Hs),
                   "parallelism": f"instances sharded round-robin over {world} GPU(s)"},
        "instances_per_s": 64 / sec,
        "tile_variants": {k: v[0] for k, v in tuned.items()},
        "converged": [sum(o["converged"] for o in out) for out in outs],
        "cycles_mean": [statistics.mean(o["cycles"] for o in out) for out in outs],
        "clocks": clk,
        "batched_hessvec": ops,
    }
    print(json.dumps(line))
    return 0


def main():
    args = parse()
    if args.oracle_worker:
        return oracle_worker(json.loads(args.oracle_worker))
    if args.impl == "reference":
        return run_reference(args)
    if args.batched_ops:
        return run_batched_ops(args)
    if args.batched:
        return run_batched(args)
    if args.paper_scale:
        return run_paper_scale(args)
    if args.learned:
        return run_learned(args)
    if args.unet_kernels:
        return run_unet_kernels(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
