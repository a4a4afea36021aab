#!/usr/bin/env python
"""Benchmark: Poisson solves per second at relative residual 1e-8 on the steep
periodic 2-D wave (512 x 17 sigma grid, kh = 2, four harmonics with
a_n = a1 0.3^(n-1), a1/h = 0.08), subspace-accelerated (EWMA, k = 10, r = 0.9)
against the plain FP64 cold start, with GMRES iterations per solve.

One step = one LSERK45 time step = 5 stages, each stage the full hot path:
right-hand side and Runge-Kutta updates, geometry, subspace guess (sketch
update, W = A Y, Gram, CholeskyQR2, x0 = Y z) and restarted GMRES.

Usage:  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl sawave|reference]
For N > 1 run it under torch.distributed.run: every rank advances its own
replica of the workload (the method has no exchange step across replicas).
Prints one JSON line on rank 0.
"""
import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Poisson solves/s at rel. residual 1e-8: accelerated vs plain; GMRES iters/solve"
UNIT = "solves/s"
WORKLOAD = "stokes2d_512x17_kh2_a1h0.08"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None, help="timed steps (default per workload)")
    ap.add_argument("--warmup", type=int, default=None, help="untimed warm-up steps (default per workload)")
    ap.add_argument("--impl", default="sawave", choices=["sawave", "reference"])
    ap.add_argument("--decay", type=float, default=0.9)
    ap.add_argument("--k", type=int, default=10)
    ap.add_argument("--plain-steps", type=int, default=3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-roofline-large", action="store_true")
    ap.add_argument("--n3d-roof", type=int, default=512, help="roofline_large: nx = ny of the 3-D field")
    ap.add_argument("--n2d-roof", type=int, default=65536, help="roofline_large: nx of the 2-D field (33 levels)")
    ap.add_argument("--members", type=int, default=512, help="batch512: number of instances")
    ap.add_argument("--batch-budget", type=float, default=240.0, help="batch512: seconds per phase at most")
    ap.add_argument("--clusters", default="auto",
                    help="batch512: thread blocks per member (1, 2, 4, 8, 16), or auto for the library's default "
                         "launch (the largest members on clusters beside single blocks)")
    ap.add_argument("--spinup", type=int, default=800, help="flume2048: steps from rest before timing")
    ap.add_argument("--n3d", type=int, default=256, help="bumpy3d: nx = ny (512 for the roofline size)")
    ap.add_argument("--executor", default="auto", choices=["auto", "persistent", "streamed"],
                    help="how a solve runs: auto (by size), persistent kernel, or streamed kernels")
    ap.add_argument("--workload", default="stokes512",
                    choices=["stokes512", "bumpy3d", "batch512", "flume2048", "decay_sweep", "sf_sweep"],
                    help="stokes512: the headline 512 x 17 steep wave (FP64); bumpy3d: 256 x 256 x 17 "
                         "precision form vs FP64; batch512: 512 uneven instances, batched vs one by one; "
                         "flume2048: 2048 x 17 flume over the bar with walls and relaxation zones (FP64); "
                         "decay_sweep: the headline workload with EWMA decay r in {0.8, 0.9, 0.95, 1.0}; "
                         "sf_sweep: stream-function waves over kh x steepness (200 x 20), previous solution vs "
                         "range finder vs EWMA")
    a = ap.parse_args()
    # defaults per workload, each run finishing in minutes: the headline and its
    # decay sweep 40 timed steps after 8; the 3-D field 3 after 3; the batch one
    # step after 7 (past the 30 previous-solution solves that fill the history)
    steps, warm = {"stokes512": (40, 8), "decay_sweep": (40, 8), "flume2048": (40, 8), "bumpy3d": (3, 3),
                   "batch512": (2, 0), "sf_sweep": (200, 6)}[a.workload]
    if a.steps is None:
        a.steps = steps
    if a.warmup is None:
        a.warmup = warm
    return a


def workload():
    import workloads as W
    return W.stokes_like_2d(nx=512, nz=17, kh=2.0, a1_over_h=0.08, steps=1000)


N_INIT_STEPS = 6   # the paper's warm-up of the subspace method: 6 steps on the previous solution (Sec. 5.1)


def solver_kw(args, guess):
    return dict(restart=20, max_restarts=500, tol=1e-8, guess=guess, k=args.k, decay=args.decay,
                n_init_solves=5 * N_INIT_STEPS, seed=2511, executor=getattr(args, "executor", "auto"))


def cpu_model():
    """CPU model name of this host (lscpu, else /proc/cpuinfo)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        for ln in open("/proc/cpuinfo"):
            if ln.lower().startswith(("model name", "cpu part")):
                return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    return None


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.idx)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# CPU baseline: the oracle as it stands, serial, on a bounded sample
# ---------------------------------------------------------------------------
def oracle_run(args, warm_steps, timed_steps, budget_s=None):
    """The serial oracle on the benchmark's trajectory: warm_steps untimed
    steps (history fill included), then up to timed_steps timed steps."""
    import oracle as O
    import workloads as W
    wl = workload()
    kw = solver_kw(args, "ewma")
    kw.pop("executor", None)   # how the library runs a solve; the oracle has one way
    P = O.OracleProblem(wl["nx"], 1, wl["nz"], wl["lx"], 0.0, wl["h"], **kw)
    st = W.state_arrays(wl)
    phys = (wl["g"], wl["rho"], wl["dt"])
    for _ in range(warm_steps):
        for i in range(1, 6):
            P.stage(phys, i, st)
    its, n, t0 = 0, 0, time.perf_counter()
    for s in range(timed_steps):
        for i in range(1, 6):
            _, stt, _ = P.stage(phys, i, st)
            its += stt["iterations"]
            n += 1
        if budget_s is not None and time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    return n / dt, its / max(n, 1), n, dt


def _oracle_worker(a):
    ns, warm, timed, budget = a
    return oracle_run(argparse.Namespace(**ns), warm, timed, budget_s=budget)


def oracle_all_cores(args, warm_steps, timed_steps, budget_s):
    """The serial oracle as one independent replica per host core (spawned
    processes, no GPU in them): aggregate solves/s of the host."""
    import multiprocessing as mp
    n = os.cpu_count() or 1
    ns = {"k": args.k, "decay": args.decay, "executor": "auto"}
    ctx = mp.get_context("spawn")
    t0 = time.perf_counter()
    with ctx.Pool(n) as pool:
        res = pool.map(_oracle_worker, [(ns, warm_steps, timed_steps, budget_s)] * n)
    wall = time.perf_counter() - t0
    rate = sum(r[0] for r in res)
    return {"value": rate, "unit": UNIT, "cores": n, "processes": n, "cpu_model": cpu_model(),
            "iters_per_solve": statistics.mean(r[1] for r in res), "solves": int(sum(r[2] for r in res)),
            "wall_s": wall, "kind": "oracle",
            "sample": "%d independent replicas of the serial oracle, one per core, each %d untimed steps then "
                      "up to %d timed steps (stopped after %.0f s)" % (n, warm_steps, timed_steps, budget_s)}


def reference_arm(args, rank):
    if rank != 0:
        return
    warm = N_INIT_STEPS + args.warmup
    allc = oracle_all_cores(args, warm, args.steps, 120.0)
    rate = allc["value"]
    ser_rate, ser_its, n1, dt1 = oracle_run(args, warm, args.steps, budget_s=60.0)
    line = {"metric": METRIC, "value": rate, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 5000.0 / rate, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "iters_per_solve": allc["iters_per_solve"],
            "config": {"workload": WORKLOAD, "guess": "ewma", "k": args.k, "decay": args.decay, "tol": 1e-8,
                       "restart": 20, "history_fill_steps_untimed": N_INIT_STEPS},
            "cpu_baseline": dict(allc, serial={"value": ser_rate, "cores": 1, "iters_per_solve": ser_its,
                                               "solves": n1}),
            "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def replica_value(local_ms, nsolves_per_rank, world, dist=None, device=None):
    """Whole-job solves/s of independent replicas: the slowest rank's time bounds the job."""
    import torch
    t = torch.tensor([float(local_ms)], dtype=torch.float64, device=device)
    if dist is not None and world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    total_ms = float(t.item())
    return world * nsolves_per_rank / (total_ms / 1e3), total_ms


# the sources each profiled kernel is compiled from: a DRAM figure taken by
# ncu stays valid while these files are unchanged
KERNEL_SOURCES = {
    "resident_kernel": ["resident.cu", "sw_solve.cuh", "sw_device.cuh", "sw_internal.cuh", "../../include/sawave.h"],
    "solve_kernel": ["solve_kernel.cu", "solver.cu", "sw_solve.cuh", "sw_device.cuh", "sw_internal.cuh",
                     "../../include/sawave.h"],
}


def source_hash(kernel=None):
    """SHA-256 prefix of the kernel's source files (all of csrc/ when no kernel
    is named), comments and blank lines left out, so that a change of wording
    in a comment keeps a figure measured on the same code."""
    import re
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2511_18071_gb300", "csrc")
    files = KERNEL_SOURCES.get(kernel) or sorted(os.listdir(d))
    for f in files:
        text = open(os.path.join(d, f), encoding="utf-8").read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        h.update("\n".join(ln.rstrip() for ln in text.splitlines() if ln.strip()).encode())
    return h.hexdigest()[:16]


def load_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


def profile_traffic(kernel):
    """DRAM bytes per launch from the committed ncu summary, if taken on the current sources."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        d = json.load(open(path))
    except (OSError, ValueError):
        return None
    ent = d.get(kernel)
    if not ent or ent.get("source_sha") != source_hash(kernel):
        return None
    return ent.get("dram_bytes_per_launch")


def run_steps(sw, torch, prob, nsteps, flush=None, events=None):
    h = prob.handle
    for _ in range(nsteps):
        if flush is not None:
            flush.zero_()
        if events is not None:
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
        for _ in range(5):
            sw.advance_stage(h)
        if events is not None:
            b.record()
            events.append((a, b))


def gpu_arm(args, rank, world, local_rank):
    import numpy as np
    import torch

    import __graft_entry__ as ge
    ge.build()
    import paper_2511_18071_gb300 as sw
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    dist = None
    if world > 1:
        import torch.distributed as dist
    wl = workload()
    t = lambda a: torch.tensor(np.ascontiguousarray(a), device=dev)
    # untimed before every timed window: the history fill of the subspace
    # method (N_INIT_STEPS steps on the previous solution), then the warm-up
    pre = N_INIT_STEPS + args.warmup

    def make(guess, precision="fp64"):
        P = sw.Problem(wl["nx"], 1, wl["nz"], wl["lx"], 0.0, wl["h"], precision=precision, **solver_kw(args, guess))
        sw.set_physics(P.handle, sw.Physics(wl["g"], wl["rho"], wl["dt"]))
        sw.set_state(P.handle, t(wl["u"]), None, t(wl["w"]), t(wl["eta"]))
        return P

    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # 256 MiB > L2
    # ---- accelerated (EWMA) ----
    P = make("ewma")
    run_steps(sw, torch, P, pre)
    torch.cuda.synchronize()
    s0 = sw.get_stats(P.handle)
    ph0 = sw.get_phase_times(P.handle)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    sw.enable_timing(P.handle, True)
    events = []
    vis = [v for v in os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",") if v.strip()]
    gpu_index = int(vis[local_rank]) if local_rank < len(vis) and vis[local_rank].strip().isdigit() else local_rank
    with ClockSampler(gpu_index) as clk:
        wall0 = time.perf_counter()
        run_steps(sw, torch, P, args.steps, flush=flush, events=events)
        torch.cuda.synchronize()
        wall = time.perf_counter() - wall0
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    step_ms = [a.elapsed_time(b) for a, b in events]
    total_ms = sum(step_ms)
    solve_ms, n_timed = sw.get_solve_time(P.handle)
    sw.enable_timing(P.handle, False)
    s1 = sw.get_stats(P.handle)
    ph1 = sw.get_phase_times(P.handle)
    P.close()
    nsolves = 5 * args.steps
    executor_used = {0: "auto", 1: "persistent", 2: "streamed", 3: "resident"}.get(s1.get("executor"), "?")
    value, total_ms = replica_value(total_ms, nsolves, world, dist, dev)
    its = (s1["total_iterations"] - s0["total_iterations"]) / nsolves
    mflops = s1["model_flops"] - s0["model_flops"]
    mbytes = s1["model_bytes"] - s0["model_bytes"]
    launches = s1["launches"] - s0["launches"]
    # ---- plain FP64 cold start, the previous-solution baseline and the
    # precision form: same workload, same untimed steps, same timed window ----
    base = {}
    for guess, prec in (("cold", "fp64"), ("previous", "fp64"), ("ewma", "mixed")):
        Q = make(guess, prec)
        run_steps(sw, torch, Q, pre)
        torch.cuda.synchronize()
        r = _timed_steps(sw, torch, Q, args.steps, flush)
        Q.close()
        nit = r["iters_per_solve"] * nsolves
        base[guess + "_" + prec] = {
            "value": r["value"], "iters_per_solve": r["iters_per_solve"], "ms_per_solve": r["ms_per_step"] / 5,
            "steps": args.steps,
            "phase_us_per_iteration": {k: round(v * nsolves / max(nit, 1), 2) for k, v in r["phase_us_per_solve"].items()}}
    # ---- error of every timed solve against the FP64 oracle (both forms): the
    # same runs repeated untimed (the library is deterministic: same counts),
    # each solve's system and solution recorded and re-solved by the oracle ----
    errs = {}
    for prec in ("fp64", "mixed"):
        errs[prec] = _solve_errors(sw, torch, dev, wl, make("ewma", prec), pre, args.steps)
    # ---- end to end through the host-buffer C-ABI call ----
    e2e = None
    oracle_cold = None
    if not args.no_e2e:
        R = make("ewma")
        m, ncol = R.m, R.ncol
        nrec = pre + args.steps
        rec_ep = torch.empty((nrec * 5, ncol), dtype=torch.float64, pin_memory=True)
        rec_ec = torch.empty_like(rec_ep)
        rec_b = torch.empty((nrec * 5, m), dtype=torch.float64, pin_memory=True)
        dep = torch.empty(ncol, dtype=torch.float64, device=dev)
        dec = torch.empty_like(dep)
        db = torch.empty(m, dtype=torch.float64, device=dev)
        for q in range(nrec * 5):
            sw.advance_stage(R.handle)
            sw.get_last_system(R.handle, dep, dec, db)
            rec_ep[q].copy_(dep)
            rec_ec[q].copy_(dec)
            rec_b[q].copy_(db)
        torch.cuda.synchronize()
        R.close()
        E = sw.Problem(wl["nx"], 1, wl["nz"], wl["lx"], 0.0, wl["h"], **solver_kw(args, "ewma"))
        xh = torch.empty(m, dtype=torch.float64, pin_memory=True)
        for q in range(pre * 5):
            sw.solve_poisson_host(E.handle, rec_ep[q], rec_ec[q], rec_b[q], xh)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for q in range(pre * 5, nrec * 5):
            sw.solve_poisson_host(E.handle, rec_ep[q], rec_ec[q], rec_b[q], xh)
        e2e_s = time.perf_counter() - t0
        E.close()
        if dist:
            tt = torch.tensor([e2e_s], device=dev)
            dist.all_reduce(tt, op=dist.ReduceOp.MAX)
            e2e_s = float(tt.item())
        e2e = {"value": world * nsolves / e2e_s, "unit": UNIT,
               "h2d_bytes_per_step": 5 * (2 * ncol + m) * 8, "d2h_bytes_per_step": 5 * m * 8,
               "note": "sw_solve_poisson_host on the recorded systems of the same trajectory"}
        if rank == 0:
            oracle_cold = _oracle_cold_orders(wl, [(rec_ep[q].numpy(), rec_ec[q].numpy(), rec_b[q].numpy())
                                                  for q in (pre * 5, pre * 5 + 2)])
    if rank != 0:
        return
    peaks = load_peaks()
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    # FP64 peak from unit counts and clock: 2 FP64 FMA per clock per SM (GB300), 2 flops each
    fp64_peak = sm_count * 2 * 2 * (peaks.get("sm_max_mhz", 2070.0) * 1e6) / 1e12
    achieved_tf = mflops / (solve_ms / 1e3) / 1e12 if solve_ms > 0 else None
    achieved_gbs = mbytes / (solve_ms / 1e3) / 1e9 if solve_ms > 0 else None
    traffic = profile_traffic("resident_kernel" if executor_used == "resident" else "solve_kernel")
    roof = {"kernel": "resident_kernel" if executor_used == "resident" else "solve_kernel", "bound": "alu", "achieved": achieved_tf, "peak": fp64_peak,
            "unit": "TFLOP/s", "frac": (achieved_tf / fp64_peak) if achieved_tf else None,
            "traffic": traffic, "peak_source": "FP64 2 FMA/clk/SM x %d SMs x %.0f MHz" % (sm_count, peaks.get("sm_max_mhz", 2070.0)),
            "hbm": {"achieved_gbs": achieved_gbs, "peak_gbs": peaks.get("hbm_gbs"),
                    "frac": (achieved_gbs / peaks["hbm_gbs"]) if achieved_gbs and peaks.get("hbm_gbs") else None},
            "kernel_ms_per_launch": solve_ms / max(n_timed, 1), "launches_timed": n_timed,
            "kernel_share_of_step": solve_ms / total_ms if total_ms else None,
            "note": "latency-bound at this size (9,216 unknowns, L2-resident); see roofline_large"}
    cpu = None
    if not args.no_cpu_baseline:
        rate, cits, n, dt = oracle_run(args, pre, args.steps, budget_s=20.0)
        cpu = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle", "iters_per_solve": cits,
               "cpu_model": cpu_model(),
               "sample": "%d EWMA solves of the same workload and window (%d untimed steps first), serial FP64 C "
                         "oracle (%.1f s)" % (n, pre, dt),
               "all_cores": oracle_all_cores(args, pre, args.steps, 20.0)}
    cold, prev, mixed = base["cold_fp64"], base["previous_fp64"], base["ewma_mixed"]
    if oracle_cold:
        cold["oracle_cold_start_iters"] = oracle_cold
    mixed_out = {k: mixed[k] for k in ("value", "iters_per_solve", "ms_per_solve")}
    mixed_out["error_vs_fp64_oracle"] = errs["mixed"]
    roof_large = None
    if not args.no_roofline_large:
        try:
            roof_large = roofline_large(sw, torch, dev, args.n3d_roof, peaks)
            roof_large["2d"] = roofline_large(sw, torch, dev, None, peaks, nx2d=args.n2d_roof)
        except sw.SawaveError as err:
            roof_large = {"unavailable": str(err)}
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "iters_per_solve": its, "us_per_solve": 1e3 * total_ms / nsolves,
            "plain": cold, "previous": prev, "mixed": mixed_out,
            "error_vs_fp64_oracle": errs["fp64"],
            "speedup_vs_plain": value / cold["value"] / world,
            "speedup_vs_previous": value / prev["value"] / world,
            "config": {"workload": WORKLOAD, "nx": 512, "nz": 17, "unknowns": wl["m"], "guess": "ewma", "k": args.k,
                       "decay": args.decay, "tol": 1e-8, "restart": 20, "n_init_steps": N_INIT_STEPS,
                       "history_fill_steps_untimed": N_INIT_STEPS, "dt": wl["dt"], "executor": executor_used,
                       "window": "every guess mode: %d untimed steps (history fill + warm-up), then the same %d "
                                 "timed steps" % (pre, args.steps),
                       "l2": "flushed between timed steps (256 MiB write, outside the step events)",
                       "parallelism": "replicas" if world > 1 else "single"},
            "roofline": roof, "roofline_large": roof_large, "cpu_baseline": cpu, "e2e": e2e, "clocks": clk.summary(),
            "gpu_launches": launches, "launches_per_solve": launches / nsolves, "wall_s_timed": wall,
            "phase_us_per_solve": {k: round((ph1[k] - ph0[k]) / nsolves, 2) for k in ph1}}
    print(json.dumps(line), flush=True)


def roofline_large(sw, torch, dev, n3d, peaks, nx2d=None):
    """Per-kernel roofline of the streamed executor at a bandwidth size, in the
    precision form, two stage solves, then the hot kernels of an Arnoldi step
    timed alone (sw_profile_kernels: CUDA events, L2 written between launches).
    The workload is the 3-D field (n3d x n3d x 17, bumps, 16 directional
    components) or, with nx2d, a 2-D Airy field nx2d x 33 spanning nx2d / 128
    wavelengths.  Algorithmic bytes and flops per launch follow the method's
    counts per point (FP32 inner vectors and factors; m unknowns, ncol columns,
    P levels, `off` factor slots per row off the column, half of them read per
    sweep; the in-column parts as P x P inverse blocks)."""
    import workloads as W
    if nx2d:
        wl = W.airy_2d(nx=nx2d, nz=33, kh=1.0, a_over_h=0.02, waves=max(1, nx2d // 128))
        ly, v = 0.0, None
    else:
        wl = W.bumpy_3d(nx=n3d, ny=n3d)
        ly = wl["ly"]
    t0 = time.perf_counter()
    P = sw.Problem(wl["nx"], wl["ny"], wl["nz"], wl["lx"], ly, wl["h"], precision="mixed", executor="streamed",
                   restart=20, max_restarts=500, tol=1e-8, guess="ewma", k=10, decay=0.9, n_init_solves=30, seed=2511)
    create_s = time.perf_counter() - t0
    sw.set_physics(P.handle, sw.Physics(wl["g"], wl["rho"], wl["dt"]))
    t = lambda a: None if a is None else torch.tensor(a, device=dev)
    sw.set_state(P.handle, t(wl["u"]), t(wl["v"]), t(wl["w"]), t(wl["eta"]))
    for _ in range(2):
        sw.advance_stage(P.handle)
    torch.cuda.synchronize()
    st = sw.get_stats(P.handle)
    us = sw.profile_kernels(P.handle, reps=5)
    col, tx, ty = sw.autotuned_apply(P.handle)
    P.close()
    m, ncol, Pl = wl["m"], wl["nx"] * wl["ny"], wl["nz"] + 1
    if nx2d:   # flat 2-D bed: 6 factor slots off the column; 12 coefficient arrays
        off, fA, ncoef = 6, 76.0, 12
    else:      # varying 3-D bed: 84 factor slots off the column
        off, fA, ncoef = 84, 123.0, 16
    j = 10
    tp = ((Pl * (Pl + 1) // 2) + 3) & ~3   # packed triangle of an in-column inverse block (periodic grids)
    model = {   # bytes, flops per launch (class of launches)
        "apply": (8.0 * m + 4.0 * ncoef * ncol, fA * m, "alu"),
        "ilu_gather_fwd": (4.0 * (off / 2) * m + 8.0 * m, 2.0 * (off / 2) * m, "hbm"),
        "ilu_products": (2.0 * 4 * tp * ncol + 16.0 * m, 2.0 * Pl * m, "hbm"),
        "ilu_gather_bwd": (4.0 * (off / 2) * m + 6.0 * m, 2.0 * (off / 2) * m, "hbm"),
        "cgs_pass1_j10": (4.0 * (j + 2) * m, 2.0 * (j + 1) * m, "hbm"),
        "cgs_pass2_j10": (4.0 * (j + 3) * m, 4.0 * (j + 1) * m, "hbm"),
        "cgs_pass3_j10": (4.0 * (j + 3) * m, 2.0 * (j + 1) * m + 2.0 * m, "hbm"),
    }
    # the whole application: both gathers and both block-product sweeps
    parts = ("ilu_gather_fwd", "ilu_products", "ilu_gather_bwd")
    model["ilu_application"] = (sum(model[k][0] for k in parts), sum(model[k][1] for k in parts), "hbm")
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    fp32_peak = sm_count * 128 * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
    hbm = peaks.get("hbm_gbs")
    kern = {}
    for k, v in us.items():
        b, f, bound = model[k]
        gbs = b / (v * 1e-6) / 1e9 if v > 0 else None
        tfs = f / (v * 1e-6) / 1e12 if v > 0 else None
        frac = (tfs / fp32_peak) if bound == "alu" else (gbs / hbm if hbm else None)
        kern[k] = {"us_per_launch": v, "alg_bytes": b, "alg_flops": f, "gbs": gbs, "tflops": tfs, "bound": bound,
                   "frac": frac}
    dom = max((k for k in kern if k != "ilu_application"), key=lambda k: kern[k]["us_per_launch"])
    name = ("airy2d_%dx33_%dwaves" % (nx2d, max(1, nx2d // 128))) if nx2d else "bumpy3d_%dx%dx17" % (n3d, n3d)
    return {"workload": name, "unknowns": m, "precision": "mixed (FP32 inner)",
            "executor": "streamed", "create_s": create_s, "solves": 2, "iters_last_solve": st["iterations"],
            "apply_form": {"column_marching": bool(col), "tile": [tx, ty]},
            "ilu_form": "row gathers per colour, column products with packed triangular inverse blocks",
            "peaks": {"hbm_gbs": hbm, "hbm_source": "measured copy (MEASURED_PEAKS.json)",
                      "fp32_tflops": fp32_peak,
                      "fp32_source": "unit counts: %d SMs x 128 FP32 lanes x 2 flops x %.0f MHz" % (
                          sm_count, peaks.get("sm_max_mhz", 2070.0))},
            "kernels": kern, "dominant": dom,
            "timing": "sw_profile_kernels: CUDA events on its own stream, 5 launches after one untimed, "
                      "a 256 MiB buffer written before every launch (inputs from HBM)"}


def _solve_errors(sw, torch, dev, wl, P, pre, steps):
    """Run P untimed through pre + steps steps; for every solve of the last
    `steps` steps, its relative error against the oracle's solution of the same
    system (warm-started from the library's solution, tol 1e-12)."""
    import numpy as np

    import oracle as O
    run_steps(sw, torch, P, pre)
    ep = torch.empty(P.ncol, dtype=torch.float64, device=dev)
    ec = torch.empty_like(ep)
    b = torch.empty(P.m, dtype=torch.float64, device=dev)
    x = torch.empty(P.m, dtype=torch.float64, device=dev)
    recs = []
    for _ in range(5 * steps):
        sw.advance_stage(P.handle)
        sw.get_last_system(P.handle, ep, ec, b)
        sw.get_state(P.handle, pres=x)
        st = sw.get_stats(P.handle)
        recs.append((ep.cpu().numpy(), ec.cpu().numpy(), b.cpu().numpy(), x.cpu().numpy(), st["iterations"],
                     st["true_res"]))
    P.close()
    ora = O.OracleProblem(wl["nx"], 1, wl["nz"], wl["lx"], 0.0, wl["h"], restart=20, max_restarts=500, tol=1e-12)
    e = []
    for epn, ecn, bn, xn, _, _ in recs:
        ora.assemble(epn, ecn)
        xo, so, code = ora.gmres(bn, xn)
        e.append(np.linalg.norm(xn - xo) / np.linalg.norm(xo))
    e = np.array(e)
    tr = np.array([r[5] for r in recs])
    return {"max": float(e.max()), "mean": float(e.mean()), "solves": len(e), "true_res_max": float(tr.max()),
            "reference": "oracle GMRES to 1e-12 on each solve's system, started from the library's solution",
            "iters_per_solve": float(np.mean([r[4] for r in recs]))}


def _oracle_cold_orders(wl, systems):
    """Cold-start GMRES(20) iterations of the oracle on sample systems with its
    colour-column ILU order (the library's) and with the natural x-fastest order."""
    import numpy as np

    import oracle as O
    out = {}
    for name in ("colour", "natural"):
        ora = O.OracleProblem(wl["nx"], 1, wl["nz"], wl["lx"], 0.0, wl["h"], restart=20, max_restarts=500, tol=1e-8)
        if name == "natural":
            ora.build_ilu(np.arange(ora.m, dtype=np.int32))
        its = []
        for epn, ecn, bn in systems:
            ora.assemble(epn, ecn)
            _, so, _ = ora.gmres(bn)
            its.append(so["iterations"])
        out[name + "_order"] = float(np.mean(its))
    out["systems"] = len(systems)
    out["note"] = "oracle cold starts on systems of the timed window; the library uses the colour order"
    return out


def _t(torch, dev, a):
    import numpy as np
    return torch.tensor(np.ascontiguousarray(a), device=dev)


def _make(sw, torch, dev, wl, guess, precision, args):
    P = sw.Problem(wl["nx"], wl["ny"], wl["nz"], wl["lx"], wl["ly"], wl["h"], precision=precision,
                   **solver_kw(args, guess))
    sw.set_physics(P.handle, sw.Physics(wl["g"], wl["rho"], wl["dt"]))
    v = None if wl["v"] is None else _t(torch, dev, wl["v"])
    sw.set_state(P.handle, _t(torch, dev, wl["u"]), v, _t(torch, dev, wl["w"]), _t(torch, dev, wl["eta"]))
    return P


def _timed_steps(sw, torch, P, steps, flush):
    s0 = sw.get_stats(P.handle)
    ph0 = sw.get_phase_times(P.handle)
    sw.enable_timing(P.handle, True)
    ev = []
    run_steps(sw, torch, P, steps, flush=flush, events=ev)
    torch.cuda.synchronize()
    ms = sum(a.elapsed_time(b) for a, b in ev)
    kms, kn = sw.get_solve_time(P.handle)
    sw.enable_timing(P.handle, False)
    s1 = sw.get_stats(P.handle)
    ph1 = sw.get_phase_times(P.handle)
    n = 5 * steps
    return dict(value=n / (ms / 1e3), ms_per_step=ms / steps, iters_per_solve=(s1["total_iterations"] - s0["total_iterations"]) / n,
                kernel_ms=kms, kernel_launches=kn, flops=s1["model_flops"] - s0["model_flops"],
                bytes=s1["model_bytes"] - s0["model_bytes"], launches=s1["launches"] - s0["launches"],
                phase_us_per_solve={k: round((ph1[k] - ph0[k]) / n, 2) for k in ph1})


def bumpy3d_arm(args):
    """256 x 256 x 17 periodic field over bumps: precision form vs plain FP64 (EWMA both)."""
    import numpy as np
    import torch

    import __graft_entry__ as ge
    import workloads as W
    ge.build()
    import paper_2511_18071_gb300 as sw
    dev = torch.device("cuda", 0)
    wl = W.bumpy_3d(nx=args.n3d, ny=args.n3d)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    res = {}
    last = {}
    for prec in ("mixed", "fp64"):
        t0 = time.perf_counter()
        P = _make(sw, torch, dev, wl, "ewma", prec, args)
        create_s = time.perf_counter() - t0
        run_steps(sw, torch, P, args.warmup)
        torch.cuda.synchronize()
        with ClockSampler(0) as clk:
            r = _timed_steps(sw, torch, P, args.steps, flush)
        r["create_s"] = create_s
        r["clocks"] = clk.summary()
        ep = torch.empty(P.ncol, dtype=torch.float64, device=dev)
        ec = torch.empty_like(ep)
        b = torch.empty(P.m, dtype=torch.float64, device=dev)
        sw.get_last_system(P.handle, ep, ec, b)
        last[prec] = (ep, ec, b)
        res[prec] = r
        P.close()
    # error of a mixed solve against an FP64 solve of the same system, both to 1e-8
    ep, ec, b = last["mixed"]
    xs = {}
    for prec in ("mixed", "fp64"):
        Q = sw.Problem(wl["nx"], wl["ny"], wl["nz"], wl["lx"], wl["ly"], wl["h"], precision=prec,
                       **dict(solver_kw(args, "cold"), tol=1e-10))
        x = torch.zeros(Q.m, dtype=torch.float64, device=dev)
        Q.solve(ep, ec, b, x)
        torch.cuda.synchronize()
        xs[prec] = x.cpu().numpy()
        Q.close()
    err = float(np.linalg.norm(xs["mixed"] - xs["fp64"]) / np.linalg.norm(xs["fp64"]))
    peaks = load_peaks()
    mx = res["mixed"]
    ach = mx["bytes"] / (mx["kernel_ms"] / 1e3) / 1e9
    line = {"metric": METRIC, "value": mx["value"], "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": mx["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic", "iters_per_solve": mx["iters_per_solve"],
            "fp64": res["fp64"], "mixed": mx, "speedup_vs_fp64": mx["value"] / res["fp64"]["value"],
            "mixed_vs_fp64_rel_error_tol1e-10": err,
            "roofline": {"kernel": "whole precision-form solve (%s executor, every kernel of the solve)"
                                   % (args.executor if args.executor != "auto"
                                      else ("streamed" if wl["m"] > 262144 else "persistent")),
                         "bound": "hbm", "achieved": ach,
                         "peak": peaks.get("hbm_gbs"), "unit": "GB/s",
                         "frac": ach / peaks["hbm_gbs"] if peaks.get("hbm_gbs") else None, "traffic": None,
                         "note": "model bytes of the solves over their kernel time; per-kernel fractions are in "
                                 "the headline line's roofline_large"},
            "config": {"workload": "bumpy3d_%dx%dx17" % (args.n3d, args.n3d), "unknowns": wl["m"], "guess": "ewma",
                       "k": args.k,
                       "executor": args.executor,
                       "decay": args.decay, "tol": 1e-8, "restart": 20,
                       "l2": "inputs larger than L2 and flushed between timed steps"}}
    print(json.dumps(line), flush=True)


def batch512_arm(args):
    """Config 5: 512 uneven 2-D instances advanced in one batched launch per
    stage, against the same instances advanced one by one through the
    single-problem API.  Two copies of the instances start from rest at t = 0
    (the same states, so the same trajectories): the history fill (N_INIT_STEPS
    steps on the previous-solution guess) and then K EWMA steps, each phase
    timed batched on one copy and one by one on the other.  Progress goes to
    stderr; a phase stops early at --batch-budget seconds and says so."""
    import concurrent.futures as cf

    import torch

    import __graft_entry__ as ge
    import workloads as W
    ge.build()
    import paper_2511_18071_gb300 as sw
    dev = torch.device("cuda", 0)
    members = W.batch_members(n=args.members)
    prec = "mixed"
    log = lambda *a: print("[batch512 %.1fs]" % (time.perf_counter() - T0), *a, file=sys.stderr, flush=True)
    T0 = time.perf_counter()

    def make():
        with cf.ThreadPoolExecutor(max_workers=16) as ex:
            ps = list(ex.map(lambda wl: sw.Problem(wl["nx"], 1, wl["nz"], wl["lx"], 0.0, wl["h"], precision=prec,
                                                    **solver_kw(args, "ewma")), members))
        for P, wl in zip(ps, members):
            sw.set_physics(P.handle, sw.Physics(wl["g"], wl["rho"], wl["dt"]))
            sw.set_state(P.handle, _t(torch, dev, wl["u"]), None, _t(torch, dev, wl["w"]),
                         _t(torch, dev, wl["eta"]))
        return ps

    probs = make()
    single = make()
    torch.cuda.synchronize()
    create_s = time.perf_counter() - T0
    log("created 2 x %d problems" % len(probs))
    B = sw.Batch(probs)
    if args.clusters != "auto":
        B.set_cluster(int(args.clusters))
    shape = B.launch_shape()
    tile, tile_us = B.autotuned_tile()
    log("launch shape", shape, "tile", tile, tile_us)

    def phase(name, ps, nsteps, one_stage):
        it0 = sum(sw.get_stats(P.handle)["total_iterations"] for P in ps)
        t0 = time.perf_counter()
        ms, done = 0.0, 0
        for step in range(nsteps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            for _ in range(5):
                one_stage()
            b.record()
            torch.cuda.synchronize()
            ms += a.elapsed_time(b)
            done += 1
            log("%s step %d: %.1f ms" % (name, step + 1, a.elapsed_time(b)))
            if time.perf_counter() - t0 > args.batch_budget:
                log("%s: budget reached after %d of %d steps" % (name, done, nsteps))
                break
        stats = [sw.get_stats(P.handle) for P in ps]
        it1 = sum(s["total_iterations"] for s in stats)
        n = len(ps) * 5 * done
        bad = [{"member": members[i]["name"], "status": s["status"], "iterations": s["iterations"]}
               for i, s in enumerate(stats) if s["status"] != 0]
        worst = max(range(len(ps)), key=lambda i: stats[i]["iterations"])
        return {"value": n / (ms / 1e3), "ms": ms, "steps": done, "steps_asked": nsteps, "solves": n,
                "iters_per_solve": (it1 - it0) / n, "members_not_ok": len(bad), "not_ok": bad[:4],
                "last_stage_max_iters": {"member": members[worst]["name"],
                                         "iterations": stats[worst]["iterations"]}}

    def one_by_one():
        for P in single:
            sw.advance_stage(P.handle)

    with ClockSampler(0) as clk:
        fill_b = phase("fill (batched)", probs, N_INIT_STEPS, B.advance_stage)
        fill_s = phase("fill (one by one)", single, N_INIT_STEPS, one_by_one)
        ewma_b = phase("ewma (batched)", probs, args.steps, B.advance_stage)
        ewma_s = phase("ewma (one by one)", single, args.steps, one_by_one)
    B.close()
    for P in probs + single:
        P.close()
    line = {"metric": METRIC, "value": ewma_b["value"], "unit": UNIT, "n_gpus": 1, "steps": ewma_b["steps"],
            "warmup": N_INIT_STEPS, "ms_per_step": ewma_b["ms"] / max(ewma_b["steps"], 1), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "value_is": "batched solves/s over the EWMA steps after the history fill",
            "iters_per_solve": ewma_b["iters_per_solve"],
            "fill_batched": fill_b, "fill_one_by_one": fill_s, "ewma_batched": ewma_b, "ewma_one_by_one": ewma_s,
            "speedup_vs_one_by_one": ewma_b["value"] / ewma_s["value"],
            "speedup_vs_one_by_one_fill": fill_b["value"] / fill_s["value"],
            "launch": {"members_on_clusters": shape[0], "blocks_per_cluster_member": shape[1],
                       "cluster_launch_blocks": shape[2], "single_block_launch_blocks": shape[3],
                       "tile_columns": tile, "tile_us_per_batched_apply": tile_us},
            "create_s": create_s, "clocks": clk.summary(), "gpu_launches_per_stage_batched": 7,
            "config": {"workload": "batch512_uneven_2d", "instances": len(members),
                       "unknowns_total": int(sum(wl["m"] for wl in members)), "guess": "ewma", "k": args.k,
                       "decay": args.decay, "tol": 1e-8, "restart": 20, "precision": prec,
                       "history_fill_steps": N_INIT_STEPS, "points_per_wavelength": 128,
                       "one_by_one": "a second copy of the same instances from the same states, through "
                                     "sw_advance_stage (each on the executor chosen for it)"}}
    print(json.dumps(line), flush=True)


def flume2048_arm(args):
    """2048 x 17 flume over the trapezoidal bar, walls and relaxation zones: EWMA vs previous vs cold.

    The flume is spun up from rest (--spinup steps, past the ramp of the incident
    wave) with the EWMA solver; the other guesses continue from the same saved
    state and time."""
    import torch

    import __graft_entry__ as ge
    import workloads as W
    ge.build()
    import paper_2511_18071_gb300 as sw
    dev = torch.device("cuda", 0)
    wl = W.flume_2d()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def make(guess):
        P = sw.Problem(wl["nx"], 1, wl["nz"], wl["lx"], 0.0, wl["h"], walls=True, **solver_kw(args, guess))
        sw.set_physics(P.handle, sw.Physics(wl["g"], wl["rho"], wl["dt"]))
        sw.set_relaxation(P.handle, wl["relax"])
        return P

    P = make("ewma")
    sw.set_state(P.handle, _t(torch, dev, wl["u"]), None, _t(torch, dev, wl["w"]), _t(torch, dev, wl["eta"]))
    run_steps(sw, torch, P, args.spinup)
    torch.cuda.synchronize()
    u = torch.empty(P.m, dtype=torch.float64, device=dev)
    w = torch.empty_like(u)
    eta = torch.empty(P.ncol, dtype=torch.float64, device=dev)
    sw.get_state(P.handle, u=u, w=w, eta=eta)
    torch.cuda.synchronize()
    eta_max = float(eta.abs().max())
    with ClockSampler(0) as clk:
        res = {"ewma": _timed_steps(sw, torch, P, args.steps, flush)}
    P.close()
    for guess in ("previous", "cold"):
        Q = make(guess)
        sw.set_state(Q.handle, u, None, w, eta)
        sw.set_step(Q.handle, args.spinup)
        run_steps(sw, torch, Q, 1)
        torch.cuda.synchronize()
        res[guess] = _timed_steps(sw, torch, Q, args.plain_steps, flush)
        Q.close()
    ew = res["ewma"]
    slim = lambda r: {k: r[k] for k in ("value", "iters_per_solve", "ms_per_step", "phase_us_per_solve")}
    line = {"metric": METRIC, "value": ew["value"], "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.spinup, "ms_per_step": ew["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "iters_per_solve": ew["iters_per_solve"],
            "previous": slim(res["previous"]), "plain": slim(res["cold"]),
            "speedup_vs_plain": ew["value"] / res["cold"]["value"],
            "speedup_vs_previous": ew["value"] / res["previous"]["value"], "eta_max_m": eta_max,
            "clocks": clk.summary(), "phase_us_per_solve": ew["phase_us_per_solve"],
            "config": {"workload": wl["name"], "unknowns": wl["m"], "lx_m": wl["lx"], "walls": True,
                       "generation_zone_m": [wl["relax"]["gen_x0"], wl["relax"]["gen_x1"]],
                       "absorption_zone_m": [wl["relax"]["abs_x0"], wl["relax"]["abs_x1"]],
                       "wave": {"H_m": wl["relax"]["height"], "T_s": wl["relax"]["period"]}, "dt": wl["dt"],
                       "guess": "ewma", "k": args.k, "decay": args.decay, "tol": 1e-8, "restart": 20,
                       "l2": "flushed between timed steps (256 MiB write, outside the step events)"}}
    print(json.dumps(line), flush=True)


def decay_sweep_arm(args):
    """EWMA forgetting rate r on the headline trajectory (the paper's decay study)."""
    import torch

    import __graft_entry__ as ge
    ge.build()
    import paper_2511_18071_gb300 as sw
    dev = torch.device("cuda", 0)
    wl = workload()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    out = {}
    for r in (0.8, 0.9, 0.95, 1.0):
        a = argparse.Namespace(**dict(vars(args), decay=r))
        P = _make(sw, torch, dev, wl, "ewma", "fp64", a)
        run_steps(sw, torch, P, args.warmup)
        torch.cuda.synchronize()
        res = _timed_steps(sw, torch, P, args.steps, flush)
        out[str(r)] = {k: res[k] for k in ("value", "iters_per_solve", "ms_per_step")}
        P.close()
    # the randomized range finder of Algorithm 3 (K = 15 newest solutions, k = 10) on the same trajectory
    a = argparse.Namespace(**dict(vars(args), decay=0.9))
    P = sw.Problem(wl["nx"], wl["ny"], wl["nz"], wl["lx"], wl["ly"], wl["h"], precision="fp64",
                   **dict(solver_kw(a, "rrf"), history=15))
    sw.set_physics(P.handle, sw.Physics(wl["g"], wl["rho"], wl["dt"]))
    sw.set_state(P.handle, _t(torch, dev, wl["u"]), None, _t(torch, dev, wl["w"]), _t(torch, dev, wl["eta"]))
    run_steps(sw, torch, P, args.warmup)
    torch.cuda.synchronize()
    res = _timed_steps(sw, torch, P, args.steps, flush)
    rrf = {k: res[k] for k in ("value", "iters_per_solve", "ms_per_step")}
    P.close()
    best = max(out, key=lambda r: out[r]["value"])
    line = {"metric": METRIC, "value": out["0.9"]["value"], "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "by_decay": out, "best_decay": float(best), "range_finder_K15_k10": rrf,
            "config": {"workload": WORKLOAD, "guess": "ewma", "k": args.k, "tol": 1e-8, "restart": 20}}
    print(json.dumps(line), flush=True)


def sf_sweep_arm(args):
    """Stream-function waves over the kh x steepness grid of the paper's study
    (200 x 20 periodic slice, dt = 1e-4 s, six untimed steps on the previous
    solution, then the timed steps): previous solution vs the range finder
    (K = 15, k = 10, V = X Omega) vs EWMA (k = 10, r = 0.7), and both subspace
    guesses again with V = Q (rrf_q, ewma_q: the orthonormalised sketch)."""
    import torch

    import __graft_entry__ as ge
    import workloads as W
    ge.build()
    import paper_2511_18071_gb300 as sw
    dev = torch.device("cuda", 0)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    a = argparse.Namespace(**dict(vars(args), k=10, decay=0.7))
    cases = []
    tot_solves = tot_ms = 0.0
    with ClockSampler(0) as clk:
        for steep in (0.01, 0.3, 0.7):
            for kh in (0.4, 2.0, 4.0):
                wl = W.stream_function_2d(kh=kh, steepness=steep, dt=1e-4)
                row = {"kh": kh, "steepness_of_max": steep, "H_over_L": wl["height"] / wl["lx"],
                       "fourier_modes": wl["wave"].N}
                for guess in ("previous", "rrf", "ewma", "rrf_q", "ewma_q"):
                    kw = solver_kw(a, guess.replace("_q", ""))
                    if guess.startswith("rrf"):
                        kw["history"] = 15
                    if guess.endswith("_q"):
                        kw["orthonormalize"] = True   # V = Q, the optional QR step of Algorithms 3 and 4
                    P = sw.Problem(wl["nx"], 1, wl["nz"], wl["lx"], 0.0, wl["h"], precision="fp64", **kw)
                    sw.set_physics(P.handle, sw.Physics(wl["g"], wl["rho"], wl["dt"]))
                    sw.set_state(P.handle, _t(torch, dev, wl["u"]), None, _t(torch, dev, wl["w"]),
                                 _t(torch, dev, wl["eta"]))
                    run_steps(sw, torch, P, args.warmup)
                    torch.cuda.synchronize()
                    r = _timed_steps(sw, torch, P, args.steps, flush)
                    P.close()
                    row[guess] = {"iters_per_step": 5 * r["iters_per_solve"], "ms_per_step": r["ms_per_step"],
                                  "solves_per_s": r["value"]}
                    if guess == "ewma":
                        tot_solves += 5 * args.steps
                        tot_ms += r["ms_per_step"] * args.steps
                for guess in ("rrf", "ewma", "rrf_q", "ewma_q"):
                    row[guess]["iter_speedup"] = row["previous"]["iters_per_step"] / row[guess]["iters_per_step"] \
                        if row[guess]["iters_per_step"] else None
                    row[guess]["time_speedup"] = row["previous"]["ms_per_step"] / row[guess]["ms_per_step"]
                cases.append(row)
    line = {"metric": METRIC, "value": tot_solves / (tot_ms / 1e3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (stream-function waves by Fenton's method)", "clocks": clk.summary(),
            "value_is": "EWMA solves/s over all nine cases", "cases": cases,
            "config": {"workload": "sfwave2d_200x20 kh x steepness grid", "unknowns": 4200, "dt_s": 1e-4,
                       "tol": 1e-8, "restart": 20, "init_steps_previous": 6, "K": 15, "k": 10, "decay": 0.7,
                       "l2": "flushed between timed steps (256 MiB write, outside the step events)"}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.workload == "sf_sweep":
        sf_sweep_arm(args)
        return
    if args.workload == "flume2048":
        flume2048_arm(args)
        return
    if args.workload == "decay_sweep":
        decay_sweep_arm(args)
        return
    if args.workload == "bumpy3d":
        bumpy3d_arm(args)
        return
    if args.workload == "batch512":
        batch512_arm(args)
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        reference_arm(args, rank)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    gpu_arm(args, rank, world, local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
