"""Benchmark of the hypercube-queue stationary solver on one GB300 (or N replicas).

Workload (default): N=24 units, J=1000 clustered demand nodes, infinite queue,
nu log-uniform on [1,3], load 0.8 -- 2^24 = 16.8M states.  One step = load the
instance from device memory (validation + upward-rate table build), solve to a
relative global-balance residual of 1e-10 (FP32 sweeps in red-black layer order with
automatic over-relaxation, then iterative refinement: FP32 sweeps of the correction
against an FP64 base; FP64 base pass, layer scalars and residual), and write P, rho,
R, W to device memory.

Metric: state-updates/s = (2^N - 2) x sweeps / time, whole job.  Reported beside it:
time-to-1e-10-residual of plain FP64 Algorithm 1 and of the warm-started and other
precision paths on the same instance and GPU (median of several solves each), the
sweep kernels' HBM roofline, and the CPU oracle on the host cores (a bounded sample of
the same workload, plus whole N=20 solves to the same residual).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun every rank solves its own instance of the same shape (replicas;
the method has no cross-GPU exchange in this configuration).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2603_03019_gb300 import instances as I  # noqa: E402

WORKLOADS = {
    "n29": lambda seed: I.large_infinite_n24(seed, N=29),
    "n28": lambda seed: I.large_infinite_n24(seed, N=28),
    "n26": lambda seed: I.large_infinite_n24(seed, N=26),
    "n24": lambda seed: I.large_infinite_n24(seed),
    "n23": lambda seed: I.large_infinite_n24(seed, N=23),
    "n22": lambda seed: I.large_infinite_n24(seed, N=22),
    "n20": lambda seed: I.mixed_n20(seed, 0.6),
    "n10": lambda seed: I.small_loss_n10(seed),
}
# arithmetic of each precision path (the per-state sweep work; FP64 always for the
# layer scalars, the birth-death step and the residual)
DTYPE = {"fp32+ir": "f32 sweeps + f64 refinement base", "fp32+df64": "f32 + df64 sweeps",
         "fp32+fp64": "f32 + f64 sweeps", "fp64": "f64", "df64": "df64", "fp32": "f32"}
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per algorithmic byte of the
# FP32 sweep kernel, from one ncu capture of a smaller case of the same kernel (N=22);
# the bench's launch is too large to capture, so the traffic it reports is this ratio
# times its algorithmic bytes (traffic grows in proportion to the states swept), and is
# labelled as extrapolated.  None while no capture of the current kernel exists.
SWEEP_DRAM_PER_ALG_BYTE = 555.32e6 / 469.76e6
TRAFFIC_SOURCE = ("ncu --set full of one launch of 2 FP32 red-black sweeps at N=22 (the same kernel "
                  "variant: 640 threads, 14-entry high-part list, the current code): 555.3 MB of DRAM traffic for 469.8 MB "
                  "of algorithmic bytes, scaled to this launch by its algorithmic bytes")
METRIC = "N=24 time-to-1e-10 residual: warm-start+FP32 vs plain FP64; state-updates/s"
# the plain FP64 sweep's ALU ceiling: FP64 operations per state update counted by ncu
# (DFMA + DADD + DMUL thread instructions of two red-black FP64 sweeps at N=22, the same
# kernel variant), at the FP64 FMA rate measured by `bench.py --fp-rate` on this GPU type
FP64_OPS_PER_STATE = 46.98
FP64_RATE = 0.5292e12
BASE_SEED = {"n29": 3001, "n28": 3001, "n26": 3001, "n24": 3001, "n23": 3001, "n22": 3001, "n20": 2001, "n10": 1001}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="n24", choices=sorted(WORKLOADS))
    ap.add_argument("--precision", default="fp32+ir")
    ap.add_argument("--tol", type=float, default=1e-10)
    ap.add_argument("--omega", type=float, default=-1.0,
                    help="over-relaxation of the outer iteration: 1 = Algorithm 1 as printed, "
                         "negative = automatic (default)")
    ap.add_argument("--no-compare", action="store_true", help="skip the per-precision comparison")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-oracle baseline")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--batch", type=int, default=0, metavar="K",
                    help="batched workload: K deployments, N ~ U{12..18}, J=200 (one JSON line)")
    ap.add_argument("--warmstart", action="store_true",
                    help="learned warm start vs cold start on held-out N=16..22 instances (one JSON line)")
    ap.add_argument("--profile", action="store_true",
                    help="one instance load and `--sweeps` sweeps in --precision (fp32, df64, "
                         "fp64, or ir: correction sweeps after 4 FP32 sweeps), nothing else (for ncu)")
    ap.add_argument("--sweeps", type=int, default=2)
    ap.add_argument("--repeats", type=int, default=3,
                    help="solves per time-to-tolerance arm (the median is reported)")
    ap.add_argument("--des", action="store_true",
                    help="the service-distribution check of Section 5.5 on the GPU simulation: "
                         "MPRE of MRT and utilisation against the hypercube solution, 15 cases per "
                         "distribution (one JSON line)")
    ap.add_argument("--fp-rate", action="store_true",
                    help="FP64 and FP32 FMA issue rates of this GPU (the FP64 ceiling of the "
                         "FP64 sweep), one JSON line each, with the SM clocks sampled meanwhile")
    ap.add_argument("--order", default="redblack", choices=["ascending", "redblack"],
                    help="sweep order of the solve (--profile and the headline path)")
    return ap.parse_args()


def run_profile(args):
    """The smallest run that contains every kernel of the hot path once per layer."""
    import torch

    from paper_2603_03019_gb300 import hq

    inst = WORKLOADS[args.workload](BASE_SEED[args.workload])
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(device=dev)
    s = hq.Solver(inst.N, inst.J, inst.mode, inst.C, stream=stream)
    s.load(torch.tensor(inst.lam_j, device=dev), torch.tensor(inst.nu, device=dev),
           torch.tensor(inst.pref, device=dev))
    torch.cuda.synchronize()
    if args.precision == "ir":
        # correction sweeps: a short FP32 solve, then one launch of `sweeps` correction
        # sweeps against an FP64 base of its result (the second k_sweep launch)
        rc, st = s.solve(tol=0.0, tol_kind=hq.HQ_TOL_STEP, precision="fp32", max_sweeps=4,
                         check_every=4, order=args.order)
        hq.hq_profile_sweep(s.h, hq.HQ_PREC_FP32_IR, args.sweeps)
        st["sweeps_hi"] = args.sweeps
    else:
        prec = args.precision if args.precision in ("fp32", "df64", "fp64") else "df64"
        rc, st = s.solve(tol=0.0, tol_kind=hq.HQ_TOL_STEP, precision=prec, max_sweeps=args.sweeps,
                         check_every=args.sweeps, order=args.order)
    s.close()
    print(json.dumps({"profile": inst.name, "sweeps": st["sweeps_hi"], "rc": rc}))
    return 0


def reduce_over_ranks(ms: float, sweeps: float, device) -> tuple[float, float]:
    """Replicas: the job's time is the slowest rank's, its work the sum of the ranks'."""
    import torch
    import torch.distributed as dist

    tm = torch.tensor([ms], dtype=torch.float64, device=device)
    ts = torch.tensor([sweeps], dtype=torch.float64, device=device)
    dist.all_reduce(tm, op=dist.ReduceOp.MAX)
    dist.all_reduce(ts, op=dist.ReduceOp.SUM)
    return float(tm[0]), float(ts[0])


def dist_info():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"hq_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.fh,
                stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                t = [x.strip() for x in line.split(",")]
                if len(t) < 9:
                    continue
                try:
                    sm.append(float(t[1]))
                    smax.append(float(t[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, t[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def host_info() -> dict:
    """nproc and the lscpu model name of the host the oracle runs on."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.lower().startswith("model name"):
                model = ln.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    return {"nproc": os.cpu_count(), "cpu_model": model}


def layer_sample(inst, threads: int, reps: int = 1, n: int | None = None) -> dict:
    """Algorithm 1's update of one whole layer (literal inner loop) by the CPU oracle on
    the same instance, ``reps`` times: the dispatch rows of the layer below are built
    first (timed apart, as the paper times coefficient generation separately)."""
    import oracle

    N = inst.N
    n = N // 2 if n is None else n
    o = oracle.Oracle(inst, threads=threads)
    t0 = time.perf_counter()
    o.build_table(n - 1, n - 1)
    t_table = time.perf_counter() - t0
    times = []
    for _ in range(reps):
        o.init()
        t0 = time.perf_counter()
        o.update_layer(n)
        times.append(time.perf_counter() - t0)
    o.close()
    states = math.comb(N, n)
    return {"layer": n, "states": states, "seconds": times, "table_rows_seconds": t_table,
            "value": states * len(times) / sum(times)}


def cpu_baseline(inst, with_solves: bool = True) -> dict:
    """The oracle on the host cores: (a) one Algorithm-1 layer update of the benchmark
    instance, single-threaded and with OpenMP over the states of the layer on all host
    threads (the line's value is the latter); (b) whole oracle solves of the N=20,
    J=500, load 0.6 instance to the benchmark's 1e-10 relative balance residual, both
    ways, table build reported apart."""
    import oracle

    host = host_info()
    threads = oracle.max_threads()
    one = layer_sample(inst, 1)
    omp = layer_sample(inst, 0)
    out = {"value": omp["value"], "unit": "state-updates/s", "cores": threads, "kind": "oracle",
           "sample": f"one Algorithm-1 update of layer {omp['layer']} ({omp['states']} states) of "
                     f"the same N={inst.N} instance, OpenMP over the layer's states on {threads} "
                     f"threads; its dispatch rows built first ({omp['table_rows_seconds']:.1f} s, "
                     f"not timed)",
           "single_thread": {"value": one["value"], "unit": "state-updates/s", "cores": 1,
                             "seconds": one["seconds"][0]},
           **host}
    if with_solves:
        w = I.mixed_n20(2001, 0.6)
        tt = {}
        for name, th in (("openmp", 0), ("single_thread", 1)):
            r = oracle.solve_to_residual(w, 1e-10, threads=th)
            tt[name] = {"cores": threads if th == 0 else 1, "sweeps": r["sweeps"],
                        "residual": r["residual"], "seconds_iterate": round(r["seconds_iterate"], 3),
                        "seconds_table": round(r["seconds_table"], 3),
                        "state_updates_per_s": ((1 << w.N) - 2) * r["sweeps"] / r["seconds_iterate"]}
        out["time_to_tol"] = {"workload": w.name, "tol": 1e-10, "check_every": 8, **tt}
    return out


def run_reference(args):
    """The oracle as it stands on the host cores (OpenMP over the states of a layer on
    all host threads): each step one Algorithm-1 layer update of the same instance."""
    ws, rank, local = dist_info()
    if rank != 0:
        return 0
    import oracle

    inst = WORKLOADS[args.workload](BASE_SEED[args.workload])
    N = inst.N
    n = N // 2
    threads = oracle.max_threads()
    o = oracle.Oracle(inst, threads=0)
    o.build_table(n - 1, n - 1)
    times = []
    for i in range(args.warmup + args.steps):
        o.init()
        t0 = time.perf_counter()
        o.update_layer(n)
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            times.append(dt)
    o.close()
    states = math.comb(N, n)
    total = sum(times)
    value = states * len(times) / total
    host = host_info()
    sample = (f"one Algorithm-1 update of layer {n} ({states} states) of the same N={N} instance "
              f"per step, OpenMP over the layer's states on {threads} threads")
    line = {"metric": METRIC, "value": value,
            "unit": "state-updates/s", "n_gpus": ws if ws > 1 else args.gpus, "steps": args.steps,
            "warmup": args.warmup,
            "ms_per_step": 1000 * total / len(times), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": inst.name, "N": N, "J": inst.J, "mode": I.MODE_NAMES[inst.mode],
                       "sample": f"layer {n} update per step", "device": "host CPU", **host},
            "cpu_baseline": {"value": value, "unit": "state-updates/s", "cores": threads,
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "state-updates/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def run_ours(args):
    import torch

    from paper_2603_03019_gb300 import hq

    ws, rank, local = dist_info()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)
    hq.load()
    stream = torch.cuda.Stream(device=dev)
    inst = WORKLOADS[args.workload](BASE_SEED[args.workload] + 97 * rank)
    N, J = inst.N, inst.J
    lam_d = torch.tensor(inst.lam_j, device=dev)
    nu_d = torch.tensor(inst.nu, device=dev)
    pref_d = torch.tensor(inst.pref, device=dev)
    S = 1 << N
    out_P = torch.empty(S, dtype=torch.float64, device=dev)
    out_rho = torch.empty(N, dtype=torch.float64, device=dev)
    out_R = torch.empty(J * N, dtype=torch.float64, device=dev)
    out_W = torch.empty(N * J, dtype=torch.float64, device=dev)
    solver = hq.Solver(N, J, inst.mode, inst.C, stream=stream)
    prec = hq.PRECISION[args.precision]

    order = hq.ORDER[args.order]

    def opts(precision=prec, tol=args.tol, omega=args.omega, sweep_order=order, warm=hq.HQ_WARM_NONE):
        o = hq.hq_default_opts()
        o.tol = tol
        o.tol_kind = hq.HQ_TOL_RESIDUAL
        o.precision = precision
        o.check_every = 8
        o.omega = omega
        o.sweep_order = sweep_order
        o.warm_start = warm
        return o

    def step_device():
        hq.hq_load(solver.h, lam_d, nu_d, pref_d)
        rc, st = hq.hq_solve(solver.h, opts())
        hq.hq_get_stationary(solver.h, out_P)
        hq.hq_get_utilisation(solver.h, out_rho)
        hq.hq_get_response_pattern(solver.h, out_R)
        hq.hq_get_workload(solver.h, out_W)
        return rc, st

    def barrier():
        if ws > 1:
            import torch.distributed as dist

            dist.barrier()

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step_device()
        torch.cuda.synchronize()
        barrier()
        clocks = ClockSampler(local)
        clocks.start()
        hq.hq_launch_count(reset=True)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        ev0.record(stream)
        sweeps_total, stats = 0, []
        kern = {"fp32_ms": 0.0, "fp32_sweeps": 0, "hi_ms": 0.0, "hi_sweeps": 0}
        for _ in range(args.steps):
            rc, st = step_device()
            stats.append(st.as_dict())
            sweeps_total += st.sweeps_fp32 + st.sweeps_hi
            kern["fp32_ms"] += st.ms_sweeps_fp32
            kern["fp32_sweeps"] += st.sweeps_fp32
            kern["hi_ms"] += st.ms_sweeps_hi
            kern["hi_sweeps"] += st.sweeps_hi
        ev1.record(stream)
        torch.cuda.synchronize()
        launches = hq.hq_launch_count()
        clk = clocks.stop()
        barrier()
        ms = ev0.elapsed_time(ev1)
        if ws > 1:
            ms, sweeps_all = reduce_over_ranks(ms, float(sweeps_total), dev)
        else:
            sweeps_all = float(sweeps_total)
        value = (S - 2) * sweeps_all / (ms / 1000.0)

        # ---- end to end through the public API with host buffers --------------------------
        e2e = None
        if not args.no_e2e:
            lam_h = torch.tensor(inst.lam_j).pin_memory()
            nu_h = torch.tensor(inst.nu).pin_memory()
            pref_h = torch.tensor(inst.pref).pin_memory()
            P_h = torch.empty(S, dtype=torch.float64).pin_memory()
            rho_h = torch.empty(N, dtype=torch.float64).pin_memory()
            R_h = torch.empty(J * N, dtype=torch.float64).pin_memory()
            W_h = torch.empty(N * J, dtype=torch.float64).pin_memory()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            sw = 0
            for _ in range(args.steps):
                hq.hq_load(solver.h, lam_h, nu_h, pref_h)
                rc, st = hq.hq_solve(solver.h, opts())
                hq.hq_get_stationary(solver.h, P_h)
                hq.hq_get_utilisation(solver.h, rho_h)
                hq.hq_get_response_pattern(solver.h, R_h)
                hq.hq_get_workload(solver.h, W_h)
                sw += st.sweeps_fp32 + st.sweeps_hi
            torch.cuda.synchronize()
            te = time.perf_counter() - t0
            h2d = inst.lam_j.nbytes + inst.nu.nbytes + inst.pref.nbytes
            d2h = (S + N + 2 * J * N) * 8
            e2e = {"value": (S - 2) * sw * ws / te, "unit": "state-updates/s",
                   "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                   "ms_per_step": 1000 * te / args.steps}

        # ---- time to tolerance per path (same instance, same GPU, median of repeats) ---------
        compare = {}
        if not args.no_compare and rank == 0:
            hq.hq_load(solver.h, lam_d, nu_d, pref_d)
            mlp = hq.load_warmstart_model()
            hq.hq_attach_mlp(solver.h, mlp)
            RB, AS = hq.HQ_ORDER_REDBLACK, hq.HQ_ORDER_ASCENDING
            W0, WL, WA = hq.HQ_WARM_NONE, hq.HQ_WARM_MLP, hq.HQ_WARM_PRODUCT
            runs = (("fp64", "fp64", 1.0, AS, W0),                 # Algorithm 1 as printed
                    ("fp32+ir", "fp32+ir", -1.0, RB, W0),          # the headline path
                    ("warm-learned+fp32+ir", "fp32+ir", -1.0, RB, WL),
                    ("warm-analytic+fp32+ir", "fp32+ir", -1.0, RB, WA),
                    ("fp32+ir ascending", "fp32+ir", -1.0, AS, W0),
                    ("warm-learned+fp32+ir ascending", "fp32+ir", -1.0, AS, WL),
                    ("fp32+df64", "fp32+df64", -1.0, RB, W0),
                    ("fp64+sor", "fp64", -1.0, RB, W0),
                    ("fp64 redblack", "fp64", 1.0, RB, W0))
            for name, pname, om, so, warm in runs:
                if "df64" in pname and N > 28:
                    continue  # double-float tables are not kept above N = 28
                rows = []
                for _ in range(max(1, args.repeats)):
                    rc, st = hq.hq_solve(solver.h, opts(hq.PRECISION[pname], omega=om, sweep_order=so,
                                                        warm=warm))
                    rows.append(st)
                med = sorted(rows, key=lambda t: t.ms_total)[len(rows) // 2]
                compare[name] = {"ms": round(med.ms_total, 3),
                                 "ms_all": [round(t.ms_total, 3) for t in rows],
                                 "sweeps_fp32": med.sweeps_fp32, "sweeps_hi": med.sweeps_hi,
                                 "residual": med.final_residual, "omega": round(med.omega, 3),
                                 "order": "redblack" if so == RB else "ascending",
                                 "warm_used": bool(med.warm_used), "converged": bool(med.converged)}
            hq.hq_attach_mlp(solver.h, None)
            hq.hq_mlp_destroy(mlp)
            if compare["fp64"]["ms"] > 0:
                for name in compare:
                    compare[name]["speedup_vs_fp64"] = round(compare["fp64"]["ms"] / compare[name]["ms"], 3)

        # ---- roofline of the sweep kernel (the kernel that dominates the step) ----------------
        roof = None
        if rank == 0:
            peak, kind = measured_peaks()
            hq.hq_load(solver.h, lam_d, nu_d, pref_d)
            hq.hq_solve(solver.h, opts())
            # isolated launches of 8 sweeps (one launch of the solve), each precision and order
            per_prec = {}
            for oname, so in (("redblack", hq.HQ_ORDER_REDBLACK), ("ascending", hq.HQ_ORDER_ASCENDING)):
                hq.hq_solve(solver.h, opts(tol=1.0, sweep_order=so))
                for name, pc in (("fp32", hq.HQ_PREC_FP32), ("ir", hq.HQ_PREC_FP32_IR),
                                 ("df64", hq.HQ_PREC_DF64), ("fp64", hq.HQ_PREC_FP64)):
                    if name == "df64" and N > 28:
                        continue
                    msw = statistics.median(hq.hq_profile_sweep(solver.h, pc, 8) for _ in range(3))
                    nbytes = hq.hq_sweep_bytes(solver.h, pc)
                    ach = nbytes / (msw / 1000.0) / 1e9
                    per_prec[f"{name} {oname}"] = {"ms_per_sweep": round(msw, 5), "bytes_per_sweep": nbytes,
                                                   "achieved_gbs": round(ach, 1), "frac": round(ach / peak, 4)}
            # the headline figure: the FP32 sweep launches inside the timed steps (CUDA events
            # around each launch on the solver's stream), algorithmic bytes / device time
            b32 = hq.hq_sweep_bytes(solver.h, hq.HQ_PREC_FP32)
            ms32 = kern["fp32_ms"] / max(1, kern["fp32_sweeps"])
            ach = b32 / (ms32 / 1000.0) / 1e9
            traffic = (SWEEP_DRAM_PER_ALG_BYTE * 8 * b32 if SWEEP_DRAM_PER_ALG_BYTE else None)
            f64 = per_prec["fp64 redblack"]
            ceil_ms = FP64_OPS_PER_STATE * (S - 2) / FP64_RATE * 1e3
            ceil_frac = hq.hq_sweep_bytes(solver.h, hq.HQ_PREC_FP64) / (ceil_ms / 1e3) / 1e9 / peak
            roof = {"bound": "hbm",
                    "kernel": f"k_sweep<FP32>, {args.order} order: one launch = 8 sweeps of layers "
                              "1..N-1 (one grid barrier per phase)",
                    "achieved": round(ach, 1), "peak": peak, "unit": "GB/s", "frac": round(ach / peak, 4),
                    "peak_kind": f"{kind} copy bandwidth (burst)", "traffic": traffic,
                    "traffic_kind": ("extrapolated: " + TRAFFIC_SOURCE) if traffic else None,
                    "bytes_per_launch": 8 * b32, "ms_per_launch": round(8 * ms32, 4),
                    "launches_timed": kern["fp32_sweeps"] // 8,
                    "fp64_sweep": {"achieved": f64["achieved_gbs"], "frac": f64["frac"],
                                   "alu_ceiling_frac": round(ceil_frac, 4),
                                   "alu_floor_ms_per_sweep": round(ceil_ms, 4),
                                   "note": "plain FP64 sweep, isolated launches of 8 sweeps, red-black; "
                                           "ceiling = its algorithmic bytes over the time its FP64 "
                                           "operations take at the measured FP64 rate"},
                    "refinement_sweeps_in_step": {
                        "ms_per_sweep": round(kern["hi_ms"] / max(1, kern["hi_sweeps"]), 5),
                        "sweeps": kern["hi_sweeps"]},
                    "per_precision": per_prec}

    solver.close()
    if rank != 0:
        if ws > 1:
            import torch.distributed as dist

            dist.destroy_process_group()
        return 0
    cpu = None
    if not args.no_cpu and ws == 1:
        cpu = cpu_baseline(inst)
    st0 = stats[-1]
    line = {
        "metric": METRIC,
        "value": value, "unit": "state-updates/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": DTYPE.get(args.precision, args.precision),
        "data": "synthetic",
        "config": {"workload": inst.name, "N": N, "J": J, "mode": I.MODE_NAMES[inst.mode],
                   "load": round(inst.load, 4), "tol": args.tol, "precision": args.precision,
                   "omega": "automatic" if args.omega < 0 else args.omega,
                   "order": args.order, "start": "uniform (the paper's)",
                   "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU",
                   "l2": "inputs larger than L2 (FP64 table 1.8 GB, FP32 table 0.9 GB)"},
        "sweeps_per_step": {"fp32": st0["sweeps_fp32"], "hi": st0["sweeps_hi"]},
        "time_to_tol_ms": compare or None,
        "table_build_ms": st0["ms_table"],
        "gpu_launches": launches, "clocks": clk, "roofline": roof, "e2e": e2e,
        "cpu_baseline": cpu,
    }
    print(json.dumps(line))
    if ws > 1:
        import torch.distributed as dist

        dist.destroy_process_group()
    return 0


def run_batch(args):
    """K deployments with N drawn from 12..18 solved by the batched solver (one persistent
    launch per check, replayed from a captured graph, kernel variant from the autotuner)
    against the same instances solved one at a time with the same options."""
    import torch

    from paper_2603_03019_gb300 import hq

    hq.load()
    K = args.batch
    insts = I.batch_n12_18(count=K)
    stream = torch.cuda.Stream()
    solvers = [hq.Solver.for_instance(i, stream=stream) for i in insts]
    b = hq.hq_batch_create([s.h for s in solvers], stream=stream)
    # correction sweeps are a single-instance mode: batched solves refine in DF64
    bprec = "fp32+df64" if args.precision == "fp32+ir" else args.precision
    prec = hq.PRECISION[bprec]
    tuned = {}
    for name, pc in (("fp32", hq.HQ_PREC_FP32), ("df64", hq.HQ_PREC_DF64), ("fp64", hq.HQ_PREC_FP64)):
        v, ms = hq.hq_batch_tune(b, pc, 4)
        tuned[name] = {"variant": v, "ms_per_sweep": [round(float(x), 4) for x in ms]}

    def opts(omega=args.omega):
        o = hq.hq_default_opts()
        o.tol = args.tol
        o.tol_kind = hq.HQ_TOL_STEP
        o.precision = prec
        o.check_every = 8
        o.omega = omega
        return o

    for _ in range(max(1, args.warmup)):
        hq.hq_batch_solve(b, K, opts())
    times, sweeps = [], []
    for _ in range(args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rc, stats, _ = hq.hq_batch_solve(b, K, opts())
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t0)
        sweeps.append(sum(((1 << i.N) - 2) * (st["sweeps_fp32"] + st["sweeps_hi"])
                          for i, st in zip(insts, stats)))
    t_batch = min(times)
    upd = sweeps[times.index(t_batch)]
    conv = sum(st["converged"] for st in stats)
    info = hq.hq_batch_info(b)
    hq.hq_batch_destroy(b)
    # one at a time, same options (step tolerance), same GPU
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    upd1 = 0.0
    for s in solvers:
        o = opts()
        rc1, st1 = hq.hq_solve(s.h, o)
        upd1 += st1.state_updates
    torch.cuda.synchronize()
    t_one = time.perf_counter() - t0
    for s in solvers:
        s.close()
    line = {
        "metric": "batched solves: instances solved per second (N ~ U{12..18}, J=200, loss, "
                  "step tolerance), one persistent launch per check under a captured graph",
        "value": K / t_batch, "unit": "instances/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1000 * t_batch, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": bprec, "data": "synthetic",
        "config": {"workload": f"batch{K}_n12_18_j200", "instances": K, "largest_N": int(info[1]),
                   "states": int(info[2]), "tol_step": args.tol, "precision": bprec,
                   "omega": "automatic" if args.omega < 0 else args.omega},
        "state_updates_per_s": upd / t_batch, "converged": conv,
        "graph": {1: "captured graph replayed", -1: "capture refused: direct launches",
                  0: "not run"}[int(info[4])],
        "autotuner": tuned,
        "one_at_a_time": {"seconds": t_one, "instances_per_s": K / t_one,
                          "state_updates_per_s": upd1 / t_one},
        "speedup_vs_one_at_a_time": t_one / t_batch,
    }
    print(json.dumps(line))
    return 0


def run_warmstart(args):
    """Held-out instances (seeds never used in training), N = 16..22, J = 300: sweeps and
    wall time to a 1e-10 relative balance residual from the paper's uniform start, from
    the analytic product-form start (first-choice utilisations, the control) and from the
    learned start (both with their fallback), same solver, same GPU."""
    import torch

    from paper_2603_03019_gb300 import hq

    hq.load()
    m = hq.load_warmstart_model()
    rows = []
    for N in (16, 18, 20, 22):
        for k in range(2):
            inst = I.warmstart_instance(880_000 + 10 * N + k, N=N, J=300)
            s = hq.Solver.for_instance(inst)
            hq.hq_attach_mlp(s.h, m)
            res = {}
            for name, warm, analytic in (("cold", False, False), ("analytic", False, True),
                                         ("learned", True, False)):
                s.solve(tol=args.tol, precision=args.precision, warm_mlp=warm, warm_product=analytic)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                rc, st = s.solve(tol=args.tol, precision=args.precision, warm_mlp=warm,
                                 warm_product=analytic)
                torch.cuda.synchronize()
                res[name] = {"ms": 1000 * (time.perf_counter() - t0),
                             "sweeps": st["sweeps_fp32"] + st["sweeps_hi"],
                             "residual": st["final_residual"], "warm_used": st["warm_used"]}
            rows.append({"N": N, "seed": 880_000 + 10 * N + k, **res})
            s.close()
    hq.hq_mlp_destroy(m)
    cold = sum(r["cold"]["ms"] for r in rows)
    warm = sum(r["learned"]["ms"] for r in rows)
    line = {"metric": "time to 1e-10 residual, learned warm start vs cold start (held-out N=16..22)",
            "value": cold / warm, "unit": "speedup (cold time / learned time)", "n_gpus": 1,
            "higher_is_better": True, "data": "synthetic", "dtype": args.precision,
            "config": {"workload": "warmstart_heldout_n16_22_j300", "instances": len(rows),
                       "precision": args.precision, "tol": args.tol},
            "sweeps_cold": sum(r["cold"]["sweeps"] for r in rows),
            "sweeps_learned": sum(r["learned"]["sweeps"] for r in rows),
            "sweeps_analytic": sum(r["analytic"]["sweeps"] for r in rows),
            "time_ratio_analytic": cold / sum(r["analytic"]["ms"] for r in rows),
            "kept": {k: sum(r[k]["warm_used"] for r in rows) for k in ("analytic", "learned")},
            "rows": rows}
    print(json.dumps(line))
    return 0


def run_fp_rate(args):
    """Build and run the FMA-rate microbenchmark (microbench/fp_rate.cu) with the clocks
    sampled during it; prints its lines with the median SM clock and the FP64 rate per
    SM per cycle at that clock."""
    src = os.path.join(ROOT, "paper_2603_03019_gb300", "microbench", "fp_rate.cu")
    out_dir = os.path.join(ROOT, "paper_2603_03019_gb300", "_build")
    os.makedirs(out_dir, exist_ok=True)
    exe = os.path.join(out_dir, "fp_rate")
    nvcc = os.environ.get("NVCC") or "nvcc"
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", src, "-o", exe], check=True)
    clocks = ClockSampler(0)
    clocks.start()
    r = subprocess.run([exe, "20000", "40", "4"], capture_output=True, text=True)
    clk = clocks.stop()
    if r.returncode != 0:
        print(json.dumps({"fp_rate": "failed", "rc": r.returncode, "stderr": r.stderr[-400:]}))
        return r.returncode
    nsm = None
    try:
        import torch

        nsm = torch.cuda.get_device_properties(0).multi_processor_count
    except Exception:
        pass
    for ln in r.stdout.splitlines():
        d = json.loads(ln)
        d["clocks"] = clk
        if nsm and clk.get("sm_mhz"):
            d["fma_per_sm_per_clk"] = round(d["fma_per_s"] / (nsm * clk["sm_mhz"] * 1e6), 3)
        print(json.dumps(d))
    return 0


def run_des(args):
    """Section 5.5's check on synthetic inputs: for N in {8, 10, 12} and load in
    {0.1, 0.3, 0.5, 0.7, 0.9} (15 cases) and each service distribution, the GPU
    simulation's mean response time and unit utilisations against the exact loss-system
    solution (GPU, FP64, 1e-12 residual): MPRE in per cent as in the paper's Eq. for
    MPRE.  Per case 38,912 replications (256 per SM) of 1,000 calls, the first 200 not
    counted: 3.1e7 counted calls, more than the paper's 20 replications of 10^6, spread
    over enough independent replications to fill the GPU (each replication is one
    thread's sequential event loop).  The rate is taken through the public call with host
    arrays (copies and set-up included).  Beside it the oracle's simulation on one host
    core, timed on a bounded sample."""
    import torch

    import oracle
    from paper_2603_03019_gb300 import hq

    hq.load()
    kinds = ["exponential", "lognormal", "gamma5", "gamma05", "uniform"]
    reps, arr, warm = 38_912, 1_000, 200
    cases = [(N, ld) for N in (8, 10, 12) for ld in (0.1, 0.3, 0.5, 0.7, 0.9)]
    exact = {}
    for N, ld in cases:
        inst = I.des_instance(6000 + N, N=N, load=ld)
        tt = I.travel_times(inst)
        s = hq.Solver.for_instance(inst)
        s.solve(tol=1e-12, precision="fp64")
        R = s.response_pattern()
        served = R * inst.lam_j[:, None]
        exact[(N, ld)] = (inst, tt, s.utilisation(), float((served * tt).sum() / served.sum()))
        s.close()
    rows = {}
    gpu_s, calls = 0.0, 0
    for kind in kinds:
        mrt_err, util_err = [], []
        for N, ld in cases:
            inst, tt, rho, mrt = exact[(N, ld)]
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            g = hq.hq_des_simulate(N, inst.J, inst.lam_j, inst.nu, inst.pref, tt, kind, reps, arr, warm, 17)
            gpu_s += time.perf_counter() - t0
            calls += reps * arr
            e = oracle.des_summary(g["busy"], g["served"], g["lost"], g["window"], g["resp"], arr - warm)
            mrt_err.append(100 * abs(e["mrt"] - mrt) / e["mrt"])
            util_err.append(100 * float(np.mean(np.abs(e["util"] - rho) / e["util"])))
        rows[kind] = {"mpre_mrt_pct": round(float(np.mean(mrt_err)), 4),
                      "mpre_mrt_max_pct": round(float(np.max(mrt_err)), 4),
                      "mpre_util_pct": round(float(np.mean(util_err)), 4),
                      "mpre_util_max_pct": round(float(np.max(util_err)), 4)}
    # the oracle's simulation of one case on one host core, bounded sample
    inst, tt, _, _ = exact[(10, 0.5)]
    t0 = time.perf_counter()
    oracle.des_loss(inst, travel=tt, kind="lognormal", reps=8, arrivals=200_000, warmup=400, seed=17)
    cpu_s = time.perf_counter() - t0
    line = {"metric": "Section 5.5 check: MPRE of MRT and utilisation, GPU simulation vs hypercube "
                      "solution (15 cases per service distribution)",
            "value": calls / gpu_s, "unit": "simulated calls/s", "n_gpus": 1, "higher_is_better": True,
            "data": "synthetic", "dtype": "f32 variates, f64 clock",
            "config": {"workload": "des_n8_12_j71_loads0.1-0.9", "replications": reps, "calls": arr,
                       "warmup_calls": warm, "cases": len(cases)},
            "mpre": rows, "gpu_seconds": gpu_s,
            "cpu_baseline": {"value": 8 * 200_000 / cpu_s, "unit": "simulated calls/s", "cores": 1,
                             "kind": "oracle", "sample": "8 replications of 200,000 calls, N=10, load 0.5, "
                                                          "log-normal service"}}
    print(json.dumps(line))
    return 0


def main():
    args = parse()
    if args.des:
        return run_des(args)
    if args.fp_rate:
        return run_fp_rate(args)
    if args.warmstart:
        return run_warmstart(args)
    if args.batch:
        return run_batch(args)
    if args.impl == "reference":
        return run_reference(args)
    if args.profile:
        return run_profile(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
