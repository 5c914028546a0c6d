"""Benchmark of the DD-4DVar hot path on GB300 (one JSON line on stdout).

Default step (N = 1 headline): one batched evaluation of every local
functional J_s and its gradient on the large workload (2048 x 1024 grid,
1024 steps, 16 x 16 x 8 = 2048 uneven overlapping subdomains, overlap
8 points / 8 steps, recursive-filter B, 1e6 observations), FP64: initial
states x_b + V w, forward sweeps with the observation and overlap terms,
adjoint sweeps and V^T for all subdomains, 3.3e9 grid-point-steps per
evaluation.  The metric is grid-point-steps (one point of a subdomain's
extended box advanced one step forward and back through the adjoint) per
second.  Extra legs in the same line: the FP32-state path on the same
workload, and on the medium workload one outer iteration of Algorithm 1
(20 batched L-BFGS iterations + Exchange) in FP64 and FP32, time to a fixed
analysis RMSE, and the Gauss-Newton local solver.

Inputs are seeded and synthetic (module ``workloads``; the truth run and the
observation sampling use the library's own global model and H).  They stand
in for the paper's Hamburg reanalysis setup, which is not available.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import workloads  # noqa: E402

METRIC = "fwd+adjoint grid-point-steps/s; time-to-analysis at fixed RMSE vs FP64 path"
UNIT = "grid-point-steps/s"

# Algorithmic arithmetic per pt-step, counted from the formulas the kernels
# evaluate (add, sub, mul = 1 flop; an FMA = 2): one RHS = 35 flops; forward
# RK3 step = 3 RHS + stage combinations = 141; adjoint step = 2 recomputed
# stages (91) + 3 transposed-Jacobian products (64 each) + combinations (36)
# = 319.  Algorithmic HBM bytes per pt-step: the forward stores the new state
# (3 values), the adjoint loads it back (3 values).
FLOPS = {"forward": 141.0, "adjoint": 319.0}
VALUES_PER_PTSTEP = {"forward": 3.0, "adjoint": 3.0}
# With stored stage states the forward also stores x1, x2 (6 values) and the
# adjoint loads them instead of recomputing two stages (2 RHS + 21 = 91 flops).
FLOPS_STORED = {"forward": 141.0, "adjoint": 228.0}
VALUES_STORED = {"forward": 9.0, "adjoint": 9.0}
# With x1 alone stored (for a share f of the pt-steps) the adjoint skips the
# first stage there (one RHS + 3 FMAs = 41 flops) and both sweeps move 3 more
# values per pt-step.
FLOPS_X1_STAGE = 41.0
# FP64 on GB300: 2 FMA / clock / SM (the nominal 1.25 TFLOP/s over 152 SMs at
# 2070 MHz); FP32: 128 FMA lanes / SM.
N_SM = 152
FP64_FLOP_PER_CLK_SM = 4.0
FP32_FLOP_PER_CLK_SM = 256.0


def aggregate_ranks(ms: float, pts: float, device: str):
    """Max over ranks of the elapsed time and sum over ranks of the work
    (replicas: the only collectives, none on the data path)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return ms, pts
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    p = torch.tensor([pts], dtype=torch.float64, device=device)
    dist.all_reduce(p, op=dist.ReduceOp.SUM)
    return float(t.item()), float(p.item())


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(prefix=f"dd4dv_clocks_gpu{self.gpu}_", suffix=".csv")
            self.f = os.fdopen(fd, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if not self.proc or not self.path or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        self.path = None
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in rows for n, v in zip(names, r[5:9]) if v.lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


def build_problem(wl, precision, stream, inputs=None, shape="", ckpt_k=0):
    """Library context with truth run, synthetic observations and decomposition."""
    import paper_2205_06649_gb300 as dd
    inp = inputs if inputs is not None else workloads.generate(wl)
    ctx = dd.Context(wl.nlon, wl.nlat, inp["dt"], wl.nsteps, precision=precision,
                     h_ref=workloads.H_REF, stream=stream)
    import torch
    # truth run and H(truth) on the device; the trajectory is freed afterwards
    # (the large workload's is 52 GB)
    truth_traj = ctx.forward(torch.as_tensor(inp["x_t0"], device="cuda"))
    hx = ctx.observe(truth_traj, inp["obs_level"], inp["obs_var"], inp["obs_fi"], inp["obs_fj"]).cpu().numpy()
    del truth_traj
    torch.cuda.empty_cache()
    truth = inp["x_t0"][None]
    so = np.asarray(wl.sigma_o)[inp["obs_var"]]
    y = hx + so * inp["obs_noise"]
    ctx.set_background(inp["x_b0"])
    ctx.set_background_error(wl.sigma_b, wl.corr_len, wl.rf_passes)
    ctx.set_observations(inp["obs_level"], inp["obs_var"], inp["obs_fi"], inp["obs_fj"], y, so)
    ctx.set_decomposition(wl.P1, wl.P2, wl.Q, wl.o_lon, wl.o_lat, wl.o_t, inp["lon_cuts"],
                          inp["lat_cuts"], inp["t_cuts"], mu=wl.mu, lam=wl.lam,
                          cluster=-1 if not shape else 0, ckpt_k=ckpt_k)
    if shape == "model":   # the library's model-based launch shape, no autotuning
        pass
    elif shape:
        v = [int(x) for x in shape.split(",")]
        cf, tf, ca, ta, sg = v[:5]
        vf, va = (v[5], v[6]) if len(v) >= 7 else (0, 0)
        ctx.set_sweep_variant(vf, va)
        ctx.set_sweep_config((cf, tf), (ca, ta), bool(sg))
    return ctx, inp, truth, (inp["obs_level"], inp["obs_var"], inp["obs_fi"], inp["obs_fj"], y, so)


def solver_for(wl):
    import paper_2205_06649_gb300 as dd
    return dd.solver_defaults(lbfgs_m=wl.lbfgs_m, max_local_iters=wl.local_iters,
                              max_outer=wl.max_outer)


def timed_steps(ctx, solver, steps, zeros_dev, stream, torch):
    """K outer iterations from the start point, CUDA events on the library stream."""
    from paper_2205_06649_gb300 import _abi
    stats = _abi.dd4dv_stats()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    l0 = ctx.launch_count()
    ev0.record(stream)
    for _ in range(steps):
        ctx.set_controls(zeros_dev)
        ctx.reset_exchange()
        ctx.outer_step(solver, stats)
    ev1.record(stream)
    ev1.synchronize()
    ms = ev0.elapsed_time(ev1)
    return ms, stats, ctx.launch_count() - l0


def rmse_h(x, truth0):
    return float(np.sqrt(np.mean((x[0] - truth0[0]) ** 2)))


def time_to_analysis(ctx, solver, truth0, max_outer, torch, stream, zeros_dev):
    """Cumulative device time and analysis RMSE(h) at t0 after each outer iteration."""
    from paper_2205_06649_gb300 import _abi
    ctx.set_controls(zeros_dev)
    ctx.reset_exchange()
    out = []
    tot = 0.0
    for _ in range(max_outer):
        st = _abi.dd4dv_stats()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ctx.outer_step(solver, st)
        e1.record(stream)
        e1.synchronize()
        tot += e0.elapsed_time(e1) / 1e3
        out.append((tot, rmse_h(ctx.analysis(), truth0), st.dw_inf))
        if st.dw_inf < solver.eps_outer:
            break
    return out


def profile_summary_traffic(kernel: str, src_hash: str, precision: str, workload: str = "medium"):
    """DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum)
    from a committed ncu summary of this workload's sweeps (captured on it, or
    on a smaller case and scaled to a full launch, as the summary states), if
    it was taken on the current kernel source; otherwise None."""
    import glob
    for p in sorted(glob.glob(os.path.join(ROOT, "profiles", f"sweeps_{workload}_{precision}*.md"))):
        text = open(p).read()
        h = re.search(r"sweep_source_sha256:\s*([0-9a-f]+)", text)
        m = re.search(rf"{kernel}_dram_bytes_per_launch:\s*([0-9.eE+]+)", text)
        if h and m and h.group(1) == src_hash:
            return float(m.group(1))
    return None


def source_hash():
    p = os.path.join(ROOT, "paper_2205_06649_gb300", "csrc", "sweep.cu")
    return hashlib.sha256(open(p, "rb").read()).hexdigest()[:16]


def _oracle_sample_setup(wl, inp, y, so, n_subs):
    """Oracle setup of the first n_subs subdomains of the first time window
    (index order), the rest of the workload as it is (sample mode of
    oracle.Setup: background run up to those windows' last level)."""
    import oracle
    obs = oracle.Observations(inp["obs_level"], inp["obs_var"], inp["obs_fi"], inp["obs_fj"], y, so)
    grid = oracle.Grid(wl.nlon, wl.nlat, workloads.RADIUS, workloads.GRAVITY, workloads.OMEGA,
                       workloads.LAT_MIN_DEG, workloads.LAT_MAX_DEG)
    dec = oracle.Decomposition.make(wl.nlon, wl.nlat, wl.nsteps, wl.P1, wl.P2, wl.Q, inp["lon_cuts"],
                                    inp["lat_cuts"], inp["t_cuts"], wl.o_lon, wl.o_lat, wl.o_t)
    q0 = [s.index for s in dec.subs if s.q == 0][:n_subs]
    st = oracle.Setup(grid, inp["dt"], wl.nsteps, inp["x_b0"], obs, wl.sigma_b, dec,
                      corr_len=wl.corr_len, rf_passes=wl.rf_passes, lam=wl.lam, mu=wl.mu, sample=q0)
    return st, len(dec.subs)


# subdomains the CPU sample sets up: enough for the time budget
CPU_SAMPLE_SUBS = {"large": 12, "batching": 12}


def _cpu_baseline_child(conn, wl_name, y, so, budget_s):
    """Spawned process: sets up the oracle sample while the GPU legs run,
    then, on "go", times J and grad J of the sampled subdomains (index order,
    w = 0) until the budget is used, alone on the host cores."""
    import torch
    try:
        wl = workloads.preset(wl_name)
        inp = workloads.generate(wl)
        t0 = time.perf_counter()
        st, n_all = _oracle_sample_setup(wl, inp, y, so, CPU_SAMPLE_SUBS.get(wl_name, 64))
        prev = st.background_prev()
        setup_s = time.perf_counter() - t0
        conn.send(("ready", setup_s))
        if conn.recv() != "go":
            return
        done = pts = 0
        t0 = time.perf_counter()
        for lp in st.locals:
            s = lp.sub
            lp.J_and_grad(torch.zeros(lp.nctrl, dtype=torch.float64), st.xb_traj, prev)
            done += 1
            pts += s.nx * s.ny * (s.b - s.a)
            if time.perf_counter() - t0 > budget_s:
                break
        dt = time.perf_counter() - t0
        cores = torch.get_num_threads()
        # the same oracle on one thread: the first sampled subdomain
        torch.set_num_threads(1)
        lp = st.locals[0]
        t1 = time.perf_counter()
        lp.J_and_grad(torch.zeros(lp.nctrl, dtype=torch.float64), st.xb_traj, prev)
        dt1 = time.perf_counter() - t1
        pts1 = lp.sub.nx * lp.sub.ny * (lp.sub.b - lp.sub.a)
        conn.send({"value": pts / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
                   "sample": f"J and grad J at w = 0 of {done} of the {n_all} subdomains (the first of "
                             f"the first time window, index order), {pts} pt-steps in {dt:.1f} s; "
                             f"FP64 PyTorch-CPU oracle, autograd adjoint; set up in {setup_s:.0f} s "
                             f"beside the GPU legs, timed alone",
                   "single_thread": {"value": pts1 / dt1, "unit": UNIT, "cores": 1,
                                     "sample": f"the first of those subdomains, {pts1} pt-steps in "
                                               f"{dt1:.1f} s"}})
    except Exception as e:   # reported in the line, never fatal to the GPU measurement
        conn.send({"value": None, "unit": UNIT, "cores": None, "kind": "oracle",
                   "sample": f"failed: {type(e).__name__}: {e}"})


class CpuBaseline:
    """The CPU oracle leg, run in a spawned process (it never touches CUDA)."""

    def __init__(self, wl_name, y, so, budget_s=20.0):
        import multiprocessing as mp
        ctx = mp.get_context("spawn")
        self.conn, child = ctx.Pipe()
        self.proc = ctx.Process(target=_cpu_baseline_child, args=(child, wl_name, y, so, budget_s),
                                daemon=True)
        self.proc.start()

    def result(self, timeout_s=900.0):
        try:
            if not self.conn.poll(timeout_s):
                return {"value": None, "kind": "oracle", "sample": "set-up did not finish in time"}
            msg = self.conn.recv()
            if isinstance(msg, dict):
                return msg
            self.conn.send("go")
            if not self.conn.poll(timeout_s):
                return {"value": None, "kind": "oracle", "sample": "timed sample did not finish"}
            return self.conn.recv()
        finally:
            self.proc.join(timeout=30)
            if self.proc.is_alive():
                self.proc.terminate()


def run_reference(args):
    """Reference arm: the CPU oracle on this arm's workload and metric (FP64
    J and grad J of subdomains, pt-steps/s).  Each step evaluates a bounded
    sample: the next subdomains of the first time window, one after another.
    The twin experiment's truth run and observations come from the oracle's
    own global model, up to the last level those subdomains reach."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import torch
    import oracle
    wl = workloads.preset(args.workload)
    inp = workloads.generate(wl)
    n_subs = CPU_SAMPLE_SUBS.get(args.workload, 64)
    dec = oracle.Decomposition.make(wl.nlon, wl.nlat, wl.nsteps, wl.P1, wl.P2, wl.Q, inp["lon_cuts"],
                                    inp["lat_cuts"], inp["t_cuts"], wl.o_lon, wl.o_lat, wl.o_t)
    last = max(s.b for s in dec.subs if s.q == 0)
    grid = oracle.Grid(wl.nlon, wl.nlat, workloads.RADIUS, workloads.GRAVITY, workloads.OMEGA,
                       workloads.LAT_MIN_DEG, workloads.LAT_MAX_DEG)
    with torch.no_grad():
        truth = oracle.global_forward(grid, torch.as_tensor(inp["x_t0"]), inp["dt"], last)
    so = np.asarray(wl.sigma_o)[inp["obs_var"]]
    lev = np.asarray(inp["obs_level"])
    y = np.zeros(len(lev))
    k = np.nonzero(lev <= last)[0]
    y[k] = oracle.observe(wl.nlon, truth, lev[k], np.asarray(inp["obs_var"])[k],
                          np.asarray(inp["obs_fi"])[k], np.asarray(inp["obs_fj"])[k])
    y += so * inp["obs_noise"]
    del truth
    st, n_all = _oracle_sample_setup(wl, inp, y, so, n_subs)
    prev = st.background_prev()
    per_step = 1 if wl.nlon * wl.nlat >= 512 * 256 else max(1, len(st.locals) // 8)
    k = 0
    pts_tot = 0
    t_tot = 0.0
    for it in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        pts = 0
        for _ in range(per_step):
            lp = st.locals[k % len(st.locals)]
            k += 1
            lp.J_and_grad(torch.zeros(lp.nctrl, dtype=torch.float64), st.xb_traj, prev)
            pts += lp.sub.nx * lp.sub.ny * (lp.sub.b - lp.sub.a)
        dt = time.perf_counter() - t0
        if it >= args.warmup:
            pts_tot += pts
            t_tot += dt
    value = pts_tot / t_tot
    sample = (f"each step: J and grad J at w = 0 of {per_step} of the {n_all} subdomains (next of the "
              f"first {len(st.locals)} of the first time window); FP64 PyTorch-CPU oracle, autograd adjoint")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * t_tot / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": wl_desc(wl), "precision": "fp64", "l2": "n/a (CPU)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": torch.get_num_threads(),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# Launch shapes for the large workload, the fastest of a shape search on its
# boxes (forward cluster, forward threads, adjoint cluster, adjoint threads,
# stored stage states, forward variant, adjoint variant; variant 1 = stripe
# sweep, 0 = deep-halo FP32 sweep where it applies, 2 = two-buffer stripe
# forward / four-buffer stripe adjoint): the benchmark forces them instead of
# spending ~80 evaluations of 0.4-2.6 s on tuning.  9-CTA clusters for the
# adjoint: a GPC of 18 or 20 SMs holds two of them at one CTA per SM (135 of
# 152 SMs busy), but only one 16-CTA cluster (112 SMs).  The two-buffer
# forward fits two CTAs per SM in 10- (FP64) or 12-CTA (FP32) clusters.
DEFAULT_SHAPES = {("large", 0): "10,384,9,1024,0,2,2", ("large", 1): "12,384,9,1024,1,2,1"}


def roofline_of(ctx, prec, reps=3):
    """Roofline object of the dominant sweep: durations from CUDA events
    around each sweep launch on the library stream (dd4dv_profile_sweeps),
    algorithmic flops / bytes per pt-step times the pt-steps of one launch."""
    prof = ctx.profile_sweeps(np.zeros(ctx.ctrl_total), reps=reps)
    pts_eval = ctx.pt_steps()
    kern = "adjoint" if prof["adjoint_ms"] >= prof["forward_ms"] else "forward"
    t_k = prof[f"{kern}_ms"] / 1e3
    peaks, peaks_kind = measured_peaks()
    sm_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    tsize = 8 if prec == 0 else 4
    cfg = ctx.sweep_config()
    stored = cfg["stored_stages"]
    fl = dict(FLOPS_STORED if stored else FLOPS)
    vals = dict(VALUES_STORED if stored else VALUES_PER_PTSTEP)
    x1 = 0.0 if stored else cfg["x1_stored"]["pt_step_share"]
    if x1 > 0.0:
        fl["adjoint"] -= FLOPS_X1_STAGE * x1
        vals = {k: v + 3.0 * x1 for k, v in vals.items()}
    flops = fl[kern] * pts_eval / t_k
    bytes_ = vals[kern] * tsize * pts_eval / t_k
    hbm_peak = float(peaks["hbm_gbs"]) * 1e9
    per_clk = FP64_FLOP_PER_CLK_SM if prec == 0 else FP32_FLOP_PER_CLK_SM
    alu_peak = N_SM * per_clk * sm_mhz * 1e6
    alu_frac = flops / alu_peak
    hbm_frac = bytes_ / hbm_peak
    wl_tag = getattr(ctx, "_bench_workload", "medium")
    traffic = profile_summary_traffic(kern, source_hash(), "fp64" if prec == 0 else "fp32", wl_tag)
    if alu_frac >= hbm_frac:
        roof = {"bound": "alu", "achieved": flops / 1e12, "peak": alu_peak / 1e12, "unit": "TFLOP/s",
                "frac": alu_frac, "traffic": traffic, "kernel": f"{kern} sweep",
                "peak_source": f"derived: {N_SM} SMs x {per_clk:.0f} {'FP64' if prec == 0 else 'FP32'} "
                               f"flop/clk x {sm_mhz:.0f} MHz",
                "hbm_frac_of_" + peaks_kind: hbm_frac}
    else:
        roof = {"bound": "hbm", "achieved": bytes_ / 1e9, "peak": hbm_peak / 1e9, "unit": "GB/s",
                "frac": hbm_frac, "traffic": traffic, "kernel": f"{kern} sweep",
                "peak_source": f"hbm_gbs of {peaks_kind}", "alu_frac": alu_frac}
    roof["kernel_ms"] = prof[f"{kern}_ms"]
    roof["pt_steps_per_launch"] = pts_eval
    roof["algorithmic_per_pt_step"] = {"flops": fl[kern], "bytes": vals[kern] * tsize}
    roof["sweeps_ms"] = {"forward": prof["forward_ms"], "adjoint": prof["adjoint_ms"], "eval": prof["eval_ms"]}
    return roof


def timed_evals(ctx, w, steps, stream, torch):
    """steps batched J and grad J evaluations of every subdomain at the
    device-resident controls w, CUDA events on the library stream."""
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    l0 = ctx.launch_count()
    e0.record(stream)
    for _ in range(steps):
        ctx.eval(w)
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1), ctx.launch_count() - l0


def e2e_evals(ctx, w_dev, steps, torch, pts_per_eval=None, barrier=None):
    """The same evaluations through the public C call with HOST buffers:
    each step copies the controls in from pinned host memory and J and the
    gradient out to pinned host memory (dd4dv_eval, device_ptrs = 0).
    Returns the line's e2e object and (pt-steps, seconds) of this rank."""
    import ctypes as C
    import paper_2205_06649_gb300 as dd
    w_h = torch.empty(ctx.ctrl_total, dtype=torch.float64).pin_memory()
    w_h.copy_(w_dev.cpu())
    J_h = torch.empty(ctx.n_sub, dtype=torch.float64).pin_memory()
    g_h = torch.empty(ctx.ctrl_total, dtype=torch.float64).pin_memory()
    torch.cuda.synchronize()
    if barrier:
        barrier()
    t0 = time.perf_counter()
    for _ in range(steps):
        st = dd.lib.dd4dv_eval(ctx._h, C.c_void_p(w_h.data_ptr()), C.c_void_p(J_h.data_ptr()),
                               C.c_void_p(g_h.data_ptr()), None, 0)
        if st != 0:
            raise RuntimeError(ctx.last_error())
    t = time.perf_counter() - t0
    pts = (ctx.pt_steps() if pts_per_eval is None else pts_per_eval) * steps
    return {"value": pts / t, "unit": UNIT,
            "h2d_bytes_per_step": int(ctx.ctrl_total * 8),
            "d2h_bytes_per_step": int((ctx.n_sub + ctx.ctrl_total) * 8),
            "api": "dd4dv_eval with host buffers (controls in, J and gradient out, pinned)"}, (pts, t)


def eval_leg(args, wl, prec, inp, torch, shape, e2e=False, on_obs=None, barrier=None, steps=None,
             warmup=None, transport=None):
    """One context on the workload: warm-up, timed evaluations (and
    optionally the end-to-end leg), roofline of the dominant sweep.
    on_obs(obs) runs once the observations exist; barrier() runs on both
    sides of the timed region.  steps / warmup default to the command line's;
    the end-to-end leg takes at most 5 steps (it measures a rate)."""
    steps = args.steps if steps is None else steps
    warmup = args.warmup if warmup is None else warmup
    stream = torch.cuda.Stream()
    ctx, inp, truth, obs = build_problem(wl, prec, stream.cuda_stream, inputs=inp, shape=shape,
                                         ckpt_k=args.ckpt)
    ctx._bench_workload = wl.name
    if on_obs:
        on_obs(obs)
    pts_rank = ctx.pt_steps()
    if transport is not None and transport.world > 1:
        # this rank evaluates its block of the problem's subdomains
        from paper_2205_06649_gb300 import sharded
        s0, s1, _ = sharded.owned_block(ctx, transport)
        owned = np.zeros(ctx.n_sub, dtype=np.int32)
        owned[s0:s1] = 1
        ctx.set_owned(owned)
        b = np.asarray(ctx.boxes).astype(np.int64)
        pts_rank = int(np.sum(b[s0:s1, 1] * b[s0:s1, 3] * (b[s0:s1, 5] - b[s0:s1, 4])))
    rng = np.random.default_rng(0)
    w = torch.tensor(0.3 * rng.standard_normal(ctx.ctrl_total), device="cuda")
    for _ in range(warmup):
        ctx.eval(w)
    torch.cuda.synchronize()
    if barrier:
        barrier()
    with ClockSampler(torch.cuda.current_device()) as clk:
        ms, launches = timed_evals(ctx, w, steps, stream, torch)
    if barrier:
        barrier()
    out = {"ms": ms, "steps": steps, "launches": launches, "clocks": clk.summary(), "pt_steps": pts_rank,
           "n_sub": ctx.n_sub, "sweep_launch": ctx.sweep_config(),
           "traj_bytes": ctx.traj_total * (8 if prec == 0 else 4)}
    if transport is not None and transport.world > 1:
        ctx.set_owned(None)   # the roofline times the sweeps over the whole problem
    out["roofline"] = roofline_of(ctx, prec)
    if e2e:
        if transport is not None and transport.world > 1:
            ctx.set_owned(owned)
        out["e2e"], out["e2e_rank"] = e2e_evals(ctx, w, min(steps, 5), torch, pts_rank, barrier)
    ctx.destroy()
    del w
    torch.cuda.empty_cache()
    return out


def medium_extras(args, torch):
    """Medium workload legs: one outer iteration of Algorithm 1 in FP64 and
    in FP32 state, time to a fixed analysis RMSE (FP64 runs to its stopping
    test or max_outer; target = 1.01 x its final RMSE; outer-iteration counts
    reported), and the Gauss-Newton local solver."""
    import paper_2205_06649_gb300 as dd
    wl = workloads.preset("medium")
    inp = workloads.generate(wl)
    solver = solver_for(wl)
    res = {}
    ctxs = {}
    for prec in (0, 1):
        stream = torch.cuda.Stream()
        ctx, _, truth, _ = build_problem(wl, prec, stream.cuda_stream, inputs=inp)
        zeros = torch.zeros(ctx.ctrl_total, dtype=torch.float64, device="cuda")
        for _ in range(2):
            ctx.set_controls(zeros)
            ctx.reset_exchange()
            ctx.outer_step(solver)
        ms, st, launches = timed_steps(ctx, solver, args.steps, zeros, stream, torch)
        prof = ctx.profile_sweeps(np.zeros(ctx.ctrl_total), reps=5)
        res["fp64" if prec == 0 else "fp32_state"] = {
            "value": st.pt_steps / (ms / 1e3), "unit": UNIT, "ms_per_step": ms / args.steps,
            "evals_per_step": st.evals / args.steps, "gpu_launches_per_step": launches / args.steps,
            "sweep_launch": ctx.sweep_config(),
            "sweeps_ms": {"forward": prof["forward_ms"], "adjoint": prof["adjoint_ms"], "eval": prof["eval_ms"]}}
        ctxs[prec] = (ctx, stream, zeros, truth)
    ctx, stream, zeros, truth = ctxs[0]
    ctx32, stream32, zeros32, _ = ctxs[1]
    h64 = time_to_analysis(ctx, solver, truth[0], wl.max_outer, torch, stream, zeros)
    h32 = time_to_analysis(ctx32, solver, truth[0], wl.max_outer, torch, stream32, zeros32)
    target = 1.01 * h64[-1][1]
    t64 = next(t for t, r, _ in h64 if r <= target)
    t32 = next((t for t, r, _ in h32 if r <= target), None)
    res["time_to_analysis"] = {
        "rmse_h_background": rmse_h(inp["x_b0"], truth[0]),
        "rmse_h_fp64_final": h64[-1][1], "rmse_h_fp32_final": h32[-1][1],
        "target_rmse_h": target, "fp64_s": t64, "fp32_s": t32, "speedup": (t64 / t32) if t32 else None,
        "outer_fp64": len(h64), "outer_fp32": len(h32),
        "outer_to_target_fp64": next(i + 1 for i, (t, r, _) in enumerate(h64) if r <= target),
        "outer_to_target_fp32": next((i + 1 for i, (t, r, _) in enumerate(h32) if r <= target), None),
        "dw_inf_fp64": [d for _, _, d in h64]}
    ctx32.destroy()
    gn_solver = dd.solver_defaults(lbfgs_m=wl.lbfgs_m, max_local_iters=wl.local_iters,
                                   max_outer=wl.max_outer, local_solver=1, gn_iters=3,
                                   cg_iters=10, cg_tol=1e-6)
    for _ in range(2):
        ctx.set_controls(zeros)
        ctx.reset_exchange()
        ctx.outer_step(gn_solver)
    ms_gn, st_gn, _ = timed_steps(ctx, gn_solver, args.steps, zeros, stream, torch)
    hgn = time_to_analysis(ctx, gn_solver, truth[0], wl.max_outer, torch, stream, zeros)
    tgn = next((t for t, r, _ in hgn if r <= target), None)
    res["gauss_newton"] = {
        "settings": {"gn_iters": 3, "cg_iters": 10, "cg_tol": 1e-6},
        "value": st_gn.pt_steps / (ms_gn / 1e3), "unit": UNIT, "ms_per_step": ms_gn / args.steps,
        "rmse_h_final": hgn[-1][1], "s_to_target": tgn, "outer": len(hgn),
        "speedup_vs_lbfgs_fp64": (t64 / tgn) if tgn else None}
    ctx.destroy()
    torch.cuda.empty_cache()
    res["workload"] = wl_desc(wl)
    return res


# Weak-scaling experiment of Sec. 7 (Table 3): QP spatial subdomains whose
# extended boxes are n_loc x n_loc = 32 x 32 points (Eq. nlocx: core 24 plus
# an overlap of 4 on each side; the wall blocks take a core of 28), problem
# size 3 n_loc^2 QP.
SCALEUP_LAYOUT = {2: (2, 1), 4: (2, 2), 8: (4, 2), 16: (4, 4), 32: (8, 4), 64: (8, 8)}


def scaleup_workloads(qp, nsteps=16):
    """(decomposed workload, undecomposed workload, lon_cuts, lat_cuts) of one
    global problem: a 24 P1 x (24 P2 + 8) grid, nsteps steps, one time
    window, QP = P1 x P2 spatial subdomains with 32 x 32 extended boxes;
    observations and B as in the small workload."""
    P1, P2 = SCALEUP_LAYOUT[qp]
    nlon, nlat = 24 * P1, 24 * P2 + 8
    lon_cuts = [24 * k for k in range(P1 + 1)]
    lat_cuts = [0] + [4 + 24 * k for k in range(1, P2)] + [nlat] if P2 > 1 else [0, nlat]
    base = workloads.preset("small").replace(
        name=f"scaleup_qp{qp}", nlon=nlon, nlat=nlat, nsteps=nsteps, P1=P1, P2=P2, Q=1,
        o_lon=4, o_lat=4, o_t=0)
    return base, base.replace(name=f"scaleup_qp{qp}_undecomposed", P1=1, P2=1), lon_cuts, lat_cuts


def scaleup_rows(torch, steps, warmup, autotune=True, precision=0):
    """Measured scale-up of one outer iteration (Sec. 6-7, Eq. measurscale,
    Table 3), read as Sc_1,QP = T(undecomposed problem of size 3 n_loc^2 QP)
    / T(the same problem in QP subdomains), both on this GPU (all subdomains
    of one problem in one launch per sweep), both in the given precision
    (0 FP64, 1 FP32 state).  In FP64 the QP = 64 undecomposed box (192 x 200
    points) fits no cluster's shared memory; in FP32 it does."""
    import paper_2205_06649_gb300 as dd
    rows = []
    for qp in sorted(SCALEUP_LAYOUT):
        times = {}
        wl_dd, wl_1, lon_cuts, lat_cuts = scaleup_workloads(qp)
        for wl in (wl_dd, wl_1):
            stream = torch.cuda.Stream()
            inp = workloads.generate(wl)
            if wl.P1 > 1:
                inp["lon_cuts"] = np.asarray(lon_cuts)
                inp["lat_cuts"] = np.asarray(lat_cuts)
            try:
                ctx, inp, truth, obs = build_problem(wl, precision, stream.cuda_stream, inputs=inp,
                                                     shape="" if autotune else "model")
            except dd.DD4DVError as e:   # one box larger than a 16-CTA cluster's shared memory
                times[wl.P1 * wl.P2] = (None, str(e), 0)
                continue
            solver = solver_for(wl)
            zeros = torch.zeros(ctx.ctrl_total, dtype=torch.float64, device="cuda")
            for _ in range(warmup):
                ctx.set_controls(zeros)
                ctx.reset_exchange()
                ctx.outer_step(solver)
            ms, stats, _ = timed_steps(ctx, solver, steps, zeros, stream, torch)
            times[wl.P1 * wl.P2] = (ms / steps, ctx.sweep_config(), ctx.n_sub)
            ctx.destroy()
        t1, tq = times[1][0], times[qp][0]
        sc = (t1 / tq) if (t1 and tq) else None
        rows.append({"QP": qp, "problem_size": 3 * 32 * 32 * qp, "grid": [wl_dd.nlon, wl_dd.nlat],
                     "ms_undecomposed": t1, "ms_decomposed": tq, "scale_up": sc,
                     "shape_undecomposed": times[1][1], "shape_decomposed": times[qp][1]})
        log(f"QP={qp} ({'f32' if precision else 'f64'}): T1 {t1} ms, TQP {tq} ms, Sc {sc}")
    return rows


def scaleup_mode(args, torch):
    prec = 0 if args.precision == "f64" else 1
    rows = scaleup_rows(torch, args.steps, args.warmup, precision=prec)
    print(json.dumps({"metric": "measured scale-up Sc_1,QP of one DD-4DVar outer iteration (n_loc = 32)",
                      "unit": "ratio", "higher_is_better": True, "n_gpus": 1, "steps": args.steps,
                      "warmup": args.warmup, "dtype": "f32 state" if prec else "f64", "data": "synthetic",
                      "rows": rows}), flush=True)
    return 0


def tta_mode(args, torch):
    """Time to analysis on one workload: the full outer loop (Algorithm 1)
    with the FP64 path and with the FP32-state path from the same start,
    analysis RMSE(h) at t0 after each outer iteration, and the time each path
    needs to reach 1.01 x the FP64 path's final RMSE."""
    wl = workloads.preset(args.workload)
    inp = workloads.generate(wl)
    solver = solver_for(wl)
    hist = {}
    shapes = {}
    for prec, shape in ((0, args.shape), (1, args.shape32)):
        stream = torch.cuda.Stream()
        ctx, _, truth, _ = build_problem(wl, prec, stream.cuda_stream, inputs=inp, shape=shape)
        zeros = torch.zeros(ctx.ctrl_total, dtype=torch.float64, device="cuda")
        hist[prec] = time_to_analysis(ctx, solver, truth[0], args.outer, torch, stream, zeros)
        shapes[prec] = ctx.sweep_config()
        log(f"precision {prec}: " + " ".join(f"{t:.2f}s:{r:.4f}" for t, r, _ in hist[prec]))
        ctx.destroy()
        del zeros
        torch.cuda.empty_cache()
    target = 1.01 * hist[0][-1][1]
    t64 = next(t for t, r, _ in hist[0] if r <= target)
    t32 = next((t for t, r, _ in hist[1] if r <= target), None)
    print(json.dumps({
        "metric": "time to analysis at fixed RMSE, FP32-state path vs FP64 path", "unit": "s",
        "higher_is_better": False, "n_gpus": 1, "dtype": "f64 and f32 state", "data": "synthetic",
        "config": {"workload": wl_desc(wl), "outer_iterations": args.outer,
                   "local_solver": "L-BFGS m=%d, %d iterations" % (wl.lbfgs_m, wl.local_iters),
                   "sweep_launch": {"fp64": shapes[0], "fp32": shapes[1]}},
        "rmse_h_background": rmse_h(inp["x_b0"], inp["x_t0"]),
        "history_fp64": [[t, r] for t, r, _ in hist[0]], "history_fp32": [[t, r] for t, r, _ in hist[1]],
        "target_rmse_h": target, "fp64_s": t64, "fp32_s": t32,
        "speedup": (t64 / t32) if t32 else None}), flush=True)
    return 0


def wl_desc(wl):
    return (f"{wl.name}: {wl.nlon}x{wl.nlat} grid, {wl.nsteps} steps, {wl.P1}x{wl.P2}x{wl.Q} "
            f"subdomains ({'uneven' if wl.uneven else 'equal'}), overlap {wl.o_lon} pts / {wl.o_t} steps, "
            f"{'recursive-filter B (3 cells)' if wl.corr_len > 0 else 'diagonal B'}, "
            f"obs of vars {list(wl.obs_vars)} every {wl.obs_every} steps")


def headline_line(args, wl, prec, leg, value, t_max, world, extras, cpu):
    return {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
        "scaling": "strong", "vs_baseline": None,
        "dtype": "f64" if prec == 0 else "f32", "data": "synthetic",
        "config": {"workload": wl_desc(wl), "precision": "fp64" if prec == 0 else "fp32-state",
                   "step": f"one batched J and grad J evaluation of all {leg['n_sub']} subdomains "
                           "(x_b + V w, forward sweeps with observation and overlap terms, adjoint "
                           "sweeps, V^T), controls resident in HBM",
                   "sweep_launch": leg["sweep_launch"], "pt_steps_per_eval": leg["pt_steps"],
                   "l2": f"inputs larger than L2: trajectories {leg['traj_bytes'] / 1e9:.0f} GB",
                   "parallelism": (f"subdomains sharded over {world} ranks (contiguous blocks balanced by "
                                   "pt-steps; no data-path collective within an evaluation)")
                                  if world > 1 else "single GPU"},
        "roofline": leg["roofline"], "cpu_baseline": cpu, "e2e": leg.get("e2e"), "clocks": leg["clocks"],
        "gpu_launches": int(leg["launches"]), **extras,
    }


def outer_mode(args, wl, prec, torch, world, rank, local_rank):
    """A step is one outer iteration of Algorithm 1 from the start point
    (controls 0, exchange state l = 0): 20 batched L-BFGS iterations with
    their Armijo trials, then the Exchange."""
    import torch.distributed as dist
    import paper_2205_06649_gb300 as dd
    stream = torch.cuda.Stream()
    inp = workloads.generate(wl)
    ctx, inp, truth, obs = build_problem(wl, prec, stream.cuda_stream, inputs=inp, shape=args.shape,
                                         ckpt_k=args.ckpt)
    ctx._bench_workload = wl.name
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = CpuBaseline(wl.name, obs[4], obs[5])
    solver = solver_for(wl)
    zeros = torch.zeros(ctx.ctrl_total, dtype=torch.float64, device="cuda")
    for _ in range(args.warmup):
        ctx.set_controls(zeros)
        ctx.reset_exchange()
        ctx.outer_step(solver)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    with ClockSampler(local_rank) as clk:
        ms, stats, launches = timed_steps(ctx, solver, args.steps, zeros, stream, torch)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    t_max, pts_all = aggregate_ranks(ms, float(stats.pt_steps), "cuda")
    if rank != 0:
        ctx.destroy()
        return 0
    roof = roofline_of(ctx, prec, reps=5)
    w_host = torch.zeros(ctx.ctrl_total, dtype=torch.float64).pin_memory().numpy()
    xa_host = torch.zeros(3 * wl.nlat * wl.nlon, dtype=torch.float64).pin_memory().numpy()
    from paper_2205_06649_gb300 import _abi
    st_e = _abi.dd4dv_stats()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        ctx.set_controls(w_host)
        ctx.reset_exchange()
        ctx.outer_step(solver, st_e)
        dd.lib.dd4dv_analysis(ctx._h, xa_host.ctypes.data, 0)
    torch.cuda.synchronize()
    e2e = {"value": st_e.pt_steps / (time.perf_counter() - t0), "unit": UNIT,
           "h2d_bytes_per_step": int(ctx.ctrl_total * 8), "d2h_bytes_per_step": int(3 * wl.nlat * wl.nlon * 8),
           "api": "set_controls(host) + reset_exchange + outer_step + analysis(host)"}
    leg = {"n_sub": ctx.n_sub, "sweep_launch": ctx.sweep_config(), "pt_steps": ctx.pt_steps(),
           "traj_bytes": ctx.traj_total * (8 if prec == 0 else 4), "roofline": roof, "e2e": e2e,
           "clocks": clk.summary(), "launches": launches}
    ctx.destroy()
    torch.cuda.empty_cache()
    extras = {} if args.no_extras or world > 1 else {"medium_legs": medium_extras(args, torch)}
    line = headline_line(args, wl, prec, leg, pts_all / (t_max / 1e3), t_max, world, extras,
                         cpu.result() if cpu else None)
    line["config"]["step"] = (f"one DD-4DVar outer iteration from the start point ({wl.local_iters} batched "
                              f"L-BFGS iterations over all {leg['n_sub']} subdomains + Exchange)")
    if world > 1:   # this mode runs one independent problem per rank
        line["scaling"] = "weak"
        line["config"]["parallelism"] = f"replicas x{world} (independent problems)"
    line["config"]["evals_per_step"] = stats.evals / args.steps
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="large")
    ap.add_argument("--precision", default="f64", choices=["f64", "f32"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the other-precision leg and the medium-workload legs")
    ap.add_argument("--autotune", action="store_true",
                    help="autotune the sweep launch shapes instead of the stored defaults of the workload")
    ap.add_argument("--profile-evals", type=int, default=0,
                    help="only run this many evaluations (for an ncu launch list) and exit")
    ap.add_argument("--mode", default="eval", choices=["eval", "outer", "scaleup", "tta"],
                    help="eval: a step is one batched J and grad J evaluation of all subdomains "
                         "(default); outer: a step is one outer iteration of Algorithm 1; scaleup: the "
                         "weak-scaling experiment of Table 3 (measured scale-up of one outer iteration, "
                         "QP = 2..64); tta: time to analysis of the FP64 and FP32-state paths over "
                         "--outer outer iterations")
    ap.add_argument("--outer", type=int, default=10, help="outer iterations of --mode tta")
    ap.add_argument("--shape32", default="", help="as --shape, for the FP32-state context of --mode tta")
    ap.add_argument("--ckpt", type=int, default=0, help="ckpt_k of the decomposition (0, -1 or k > 0)")
    ap.add_argument("--shape", default="",
                    help="fwd_cluster,fwd_threads,adj_cluster,adj_threads,stored_stages[,fwd_variant,"
                         "adj_variant]: force the sweep launch shapes (e.g. ones an autotuned run reported); "
                         "variants 0 = deep-halo FP32 sweep where it applies, 1 = stripe sweep")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local_rank)
    import __graft_entry__ as g
    g.build()

    if args.mode == "scaleup":
        return scaleup_mode(args, torch) if rank == 0 else 0
    if args.mode == "tta":
        return tta_mode(args, torch) if rank == 0 else 0

    wl = workloads.preset(args.workload)
    prec = 0 if args.precision == "f64" else 1
    shape = args.shape or ("" if args.autotune else DEFAULT_SHAPES.get((wl.name, prec), ""))

    if args.profile_evals:
        stream = torch.cuda.Stream()
        ctx, _, _, _ = build_problem(wl, prec, stream.cuda_stream, shape=shape, ckpt_k=args.ckpt)
        w0 = np.zeros(ctx.ctrl_total)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("evals")   # ncu --nvtx --nvtx-include "evals/" selects these
        for _ in range(args.profile_evals):
            ctx.eval(w0)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        log(f"profile run: {args.profile_evals} evaluations, shapes {ctx.sweep_config()}")
        ctx.destroy()
        return 0

    if args.mode == "outer":
        args.shape = shape
        return outer_mode(args, wl, prec, torch, world, rank, local_rank)

    inp = workloads.generate(wl)
    cpu = None

    def on_obs(obs):
        nonlocal cpu
        if rank == 0 and world == 1 and not args.no_cpu_baseline:
            cpu = CpuBaseline(wl.name, obs[4], obs[5])

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()

    transport = None
    if world > 1:
        from paper_2205_06649_gb300 import sharded
        transport = sharded.TorchDistTransport()
    leg = eval_leg(args, wl, prec, inp, torch, shape, e2e=True, on_obs=on_obs, barrier=barrier,
                   transport=transport)
    t_max, pts_all = aggregate_ranks(leg["ms"], float(leg["pt_steps"] * args.steps), "cuda")
    if world > 1:
        e_pts, e_s = leg["e2e_rank"]
        e_t, e_p = aggregate_ranks(e_s, float(e_pts), "cuda")
        leg["e2e"]["value"] = e_p / e_t
    extras = {}
    if rank == 0 and not args.no_extras and world == 1:
        other = 1 - prec
        o = eval_leg(args, wl, other, inp, torch, DEFAULT_SHAPES.get((wl.name, other), ""),
                     steps=min(args.steps, 10), warmup=min(args.warmup, 2))
        extras["fp32_state" if other == 1 else "fp64"] = {
            "value": o["pt_steps"] * o["steps"] / (o["ms"] / 1e3), "unit": UNIT,
            "ms_per_step": o["ms"] / o["steps"], "steps": o["steps"],
            "dtype": "f32 state, f64 reductions" if other == 1 else "f64",
            "sweep_launch": o["sweep_launch"], "roofline": o["roofline"], "clocks": o["clocks"]}
        extras["medium_legs"] = medium_extras(args, torch)
        extras["scaleup_table3"] = {
            "metric": "measured scale-up Sc_1,QP of one DD-4DVar outer iteration (n_loc = 32, Table 3)",
            "steps": min(args.steps, 5), "warmup": 2, "launch_shapes": "model-based (no autotuning)",
            "rows": scaleup_rows(torch, min(args.steps, 5), 2, autotune=False),
            "rows_fp32_state": scaleup_rows(torch, min(args.steps, 5), 2, autotune=False, precision=1)}
    if rank == 0:
        line = headline_line(args, wl, prec, leg, pts_all / (t_max / 1e3), t_max, world, extras,
                             cpu.result() if cpu else None)
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
