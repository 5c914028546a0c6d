"""Benchmark of the DD-4DVar hot path on GB300 (one JSON line on stdout).

A step is one outer iteration of Algorithm 1 on the medium workload (256x128
grid, 128 steps, 4x4x4 = 64 overlapping subdomains, overlap 4 points / 4
steps, recursive-filter B, 5 % of points observed in h, u, v every 8 steps):
every subdomain is put back at the start point (controls 0, exchange state
l = 0), then 20 batched L-BFGS iterations with their Armijo trials evaluate
J and grad J of all active subdomains (initial state, forward sweep,
observation and overlap terms, adjoint sweep, V^T), and the Exchange runs
(local trajectories, overlap targets, assembled boundary trajectory,
outer increment).  The metric is grid-point-steps (one point of a subdomain's
extended box advanced one step forward and back through the adjoint) per
second over all evaluations of the step.

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
    if shape:
        cf, tf, ca, ta, sg = (int(x) for x in shape.split(","))
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


def profile_summary_traffic(kernel: str, src_hash: str, precision: str):
    """DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum)
    from a committed ncu summary of the medium workload, if it was taken on the
    current kernel source; otherwise None."""
    import glob
    for p in sorted(glob.glob(os.path.join(ROOT, "profiles", f"sweeps_medium_{precision}*.md"))):
        text = open(p).read()
        h = re.search(r"sweep_source_sha256:\s*([0-9a-f]+)", text)
        m = re.search(rf"{kernel}_dram_bytes_per_launch:\s*([0-9.eE+]+)", text)
        if h and m and h.group(1) == src_hash:
            return float(m.group(1))
    return None


def source_hash():
    p = os.path.join(ROOT, "paper_2205_06649_gb300", "csrc", "sweep.cu")
    return hashlib.sha256(open(p, "rb").read()).hexdigest()[:16]


def cpu_oracle_baseline(wl, inputs, budget_s=20.0):
    """The CPU oracle as it stands, on a bounded sample of the same workload:
    J and grad J of subdomains in index order until the time budget is used."""
    import torch
    import oracle
    st, _, _ = oracle.build_setup(wl, inputs)
    B, prev = st.xb_traj, st.background_prev()
    done = 0
    pts = 0
    t0 = time.perf_counter()
    for lp in st.locals:
        s = lp.sub
        lp.J_and_grad(torch.zeros(lp.nctrl, dtype=torch.float64), B, prev)
        done += 1
        pts += s.nx * s.ny * (s.b - s.a)
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    return {"value": pts / dt, "unit": UNIT, "cores": torch.get_num_threads(), "kind": "oracle",
            "sample": f"J and grad J of {done} of {len(st.locals)} subdomains at w = 0, "
                      f"{pts} pt-steps in {dt:.1f} s (FP64 PyTorch-CPU oracle, autograd adjoint)"}


def run_reference(args):
    """Reference arm: the CPU oracle on the same workload and metric."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import torch
    import oracle
    wl = workloads.preset(args.workload)
    inp = workloads.generate(wl)
    st, _, _ = oracle.build_setup(wl, inp)
    B, prev = st.xb_traj, st.background_prev()
    per_step = max(1, len(st.locals) // 8)
    k = 0
    pts_tot = 0
    t_tot = 0.0
    for it in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        pts = 0
        for _ in range(per_step):
            lp = st.locals[k % len(st.locals)]
            k += 1
            lp.J_and_grad(torch.zeros(lp.nctrl, dtype=torch.float64), B, prev)
            pts += lp.sub.nx * lp.sub.ny * (lp.sub.b - lp.sub.a)
        dt = time.perf_counter() - t0
        if it >= args.warmup:
            pts_tot += pts
            t_tot += dt
    value = pts_tot / t_tot
    sample = (f"each step: J and grad J of {per_step} of {len(st.locals)} subdomains "
              f"(FP64 PyTorch-CPU oracle, autograd adjoint)")
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


def eval_mode(args, ctx, wl, prec, stream, torch):
    """Steps of one batched J and grad J evaluation of every subdomain
    (device-resident controls), timed with CUDA events on the library stream."""
    rng = np.random.default_rng(0)
    w = torch.tensor(0.3 * rng.standard_normal(ctx.ctrl_total), device="cuda")
    for _ in range(args.warmup):
        ctx.eval(w)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    l0 = ctx.launch_count()
    with ClockSampler(0) as clk:
        e0.record(stream)
        for _ in range(args.steps):
            ctx.eval(w)
        e1.record(stream)
        e1.synchronize()
    ms = e0.elapsed_time(e1)
    prof = ctx.profile_sweeps(np.zeros(ctx.ctrl_total), reps=3)
    line = {"metric": "fwd+adjoint grid-point-steps/s (one batched evaluation per step)",
            "value": ctx.pt_steps() * args.steps / (ms / 1e3), "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "dtype": "f64" if prec == 0 else "f32", "data": "synthetic",
            "config": {"workload": wl_desc(wl), "n_sub": ctx.n_sub, "pt_steps_per_eval": ctx.pt_steps(),
                       "sweep_launch": ctx.sweep_config(), "ckpt_k": args.ckpt},
            "sweeps_ms": {"forward": prof["forward_ms"], "adjoint": prof["adjoint_ms"]},
            "clocks": clk.summary(), "gpu_launches": ctx.launch_count() - l0}
    print(json.dumps(line), flush=True)
    ctx.destroy()
    return 0


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


def scaleup_mode(args, torch):
    import paper_2205_06649_gb300 as dd
    """Measured scale-up of one outer iteration (Sec. 6-7, Eq. measurscale,
    Table 3), read as Sc_1,QP = T(undecomposed problem of size 3 n_loc^2 QP)
    / T(the same problem in QP subdomains), both on this GPU (all subdomains
    of one problem in one launch per sweep)."""
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
                ctx, inp, truth, obs = build_problem(wl, 0, stream.cuda_stream, inputs=inp)
            except dd.DD4DVError as e:   # one box larger than a 16-CTA cluster's shared memory
                times[wl.P1 * wl.P2] = (None, str(e), 0)
                continue
            solver = solver_for(wl)
            zeros = torch.zeros(ctx.ctrl_total, dtype=torch.float64, device="cuda")
            for _ in range(args.warmup):
                ctx.set_controls(zeros)
                ctx.reset_exchange()
                ctx.outer_step(solver)
            ms, stats, _ = timed_steps(ctx, solver, args.steps, zeros, stream, torch)
            times[wl.P1 * wl.P2] = (ms / args.steps, ctx.sweep_config(), ctx.n_sub)
            ctx.destroy()
        t1, tq = times[1][0], times[qp][0]
        sc = (t1 / tq) if (t1 and tq) else None
        rows.append({"QP": qp, "problem_size": 3 * 32 * 32 * qp, "grid": [wl_dd.nlon, wl_dd.nlat],
                     "ms_undecomposed": t1, "ms_decomposed": tq,
                     "scale_up": sc, "shape_undecomposed": times[1][1], "shape_decomposed": times[qp][1]})
        log(f"QP={qp}: T1 {t1} ms, TQP {tq} ms, Sc {sc}")
    print(json.dumps({"metric": "measured scale-up Sc_1,QP of one DD-4DVar outer iteration (n_loc = 32)",
                      "unit": "ratio", "higher_is_better": True, "n_gpus": 1, "steps": args.steps,
                      "warmup": args.warmup, "dtype": "f64", "data": "synthetic", "rows": rows}), flush=True)
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


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="medium")
    ap.add_argument("--precision", default="f64", choices=["f64", "f32"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip FP32 and time-to-analysis legs")
    ap.add_argument("--profile-evals", type=int, default=0,
                    help="only run this many evaluations (for an ncu launch list) and exit")
    ap.add_argument("--mode", default="outer", choices=["outer", "eval", "scaleup", "tta"],
                    help="outer: a step is one outer iteration (default); eval: a step is one batched "
                         "J and grad J evaluation of all subdomains (for workloads too large for the "
                         "outer-iteration bench); scaleup: the weak-scaling experiment of Table 3 "
                         "(measured scale-up of one outer iteration, QP = 2..64); tta: time to analysis "
                         "of the FP64 and FP32-state paths over --outer outer iterations")
    ap.add_argument("--outer", type=int, default=10, help="outer iterations of --mode tta")
    ap.add_argument("--shape32", default="", help="as --shape, for the FP32-state context of --mode tta")
    ap.add_argument("--ckpt", type=int, default=0, help="ckpt_k of the decomposition (0, -1 or k > 0)")
    ap.add_argument("--shape", default="",
                    help="fwd_cluster,fwd_threads,adj_cluster,adj_threads,stored_stages: force the "
                         "sweep launch shapes (e.g. ones an autotuned run reported) instead of autotuning")
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
    import paper_2205_06649_gb300 as dd

    if args.mode == "scaleup":
        return scaleup_mode(args, torch) if rank == 0 else 0
    if args.mode == "tta":
        return tta_mode(args, torch) if rank == 0 else 0

    wl = workloads.preset(args.workload)
    prec = 0 if args.precision == "f64" else 1
    stream = torch.cuda.Stream()
    ctx, inp, truth, obs = build_problem(wl, prec, stream.cuda_stream, shape=args.shape, ckpt_k=args.ckpt)
    solver = solver_for(wl)
    zeros = torch.zeros(ctx.ctrl_total, dtype=torch.float64, device="cuda")

    if args.profile_evals:
        w0 = np.zeros(ctx.ctrl_total)
        for _ in range(args.profile_evals):
            ctx.eval(w0)
        torch.cuda.synchronize()
        log(f"profile run: {args.profile_evals} evaluations, cluster {ctx.cluster_size()}")
        return 0

    if args.mode == "eval":
        return eval_mode(args, ctx, wl, prec, stream, torch)

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
    value = pts_all / (t_max / 1e3)
    clocks = clk.summary()

    line = None
    if rank == 0:
        # kernel timing (CUDA events around each sweep launch, same stream)
        prof = ctx.profile_sweeps(np.zeros(ctx.ctrl_total), reps=5)
        pts_eval = ctx.pt_steps()
        kern = "adjoint" if prof["adjoint_ms"] >= prof["forward_ms"] else "forward"
        t_k = prof[f"{kern}_ms"] / 1e3
        peaks, peaks_kind = measured_peaks()
        sm_mhz = float(peaks.get("sm_max_mhz", 2070.0))
        tsize = 8 if prec == 0 else 4
        stored = ctx.sweep_config()["stored_stages"]
        fl = FLOPS_STORED if stored else FLOPS
        vals = VALUES_STORED if stored else VALUES_PER_PTSTEP
        flops = fl[kern] * pts_eval / t_k
        bytes_ = vals[kern] * tsize * pts_eval / t_k
        hbm_peak = float(peaks["hbm_gbs"]) * 1e9
        if prec == 0:
            alu_peak = N_SM * FP64_FLOP_PER_CLK_SM * sm_mhz * 1e6
        else:
            alu_peak = N_SM * FP32_FLOP_PER_CLK_SM * sm_mhz * 1e6
        alu_frac = flops / alu_peak
        hbm_frac = bytes_ / hbm_peak
        traffic = profile_summary_traffic(kern, source_hash(), "fp64" if prec == 0 else "fp32")
        if alu_frac >= hbm_frac:
            roof = {"bound": "alu", "achieved": flops / 1e12, "peak": alu_peak / 1e12, "unit": "TFLOP/s",
                    "frac": alu_frac, "traffic": traffic, "kernel": f"{kern} sweep",
                    "peak_source": f"derived: {N_SM} SMs x {FP64_FLOP_PER_CLK_SM if prec == 0 else FP32_FLOP_PER_CLK_SM:.0f} "
                                   f"flop/clk x {sm_mhz:.0f} MHz ({'FP64' if prec == 0 else 'FP32'})",
                    "hbm_frac_of_" + peaks_kind: hbm_frac}
        else:
            roof = {"bound": "hbm", "achieved": bytes_ / 1e9, "peak": hbm_peak / 1e9, "unit": "GB/s",
                    "frac": hbm_frac, "traffic": traffic, "kernel": f"{kern} sweep",
                    "peak_source": f"hbm_gbs of {peaks_kind}", "alu_frac": alu_frac}
        roof["kernel_ms"] = prof[f"{kern}_ms"]
        roof["algorithmic_per_pt_step"] = {"flops": fl[kern], "bytes": vals[kern] * tsize}
        roof["sweeps_ms"] = {"forward": prof["forward_ms"], "adjoint": prof["adjoint_ms"],
                             "eval": prof["eval_ms"]}

        # end to end through the public API with host buffers: controls in
        # (pinned host -> device), outer iteration, analysis out (device -> pinned host)
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
        t_e2e = time.perf_counter() - t0
        e2e = {"value": st_e.pt_steps / t_e2e, "unit": UNIT,
               "h2d_bytes_per_step": int(ctx.ctrl_total * 8),
               "d2h_bytes_per_step": int(3 * wl.nlat * wl.nlon * 8),
               "api": "set_controls(host) + reset_exchange + outer_step + analysis(host)"}

        extras = {}
        if not args.no_extras and world == 1:
            # FP32-state path on the same step, and time to analysis at fixed RMSE
            stream32 = torch.cuda.Stream()
            ctx32, _, _, _ = build_problem(wl, 1, stream32.cuda_stream, inputs=inp)
            zeros32 = torch.zeros(ctx32.ctrl_total, dtype=torch.float64, device="cuda")
            for _ in range(2):
                ctx32.set_controls(zeros32)
                ctx32.reset_exchange()
                ctx32.outer_step(solver)
            ms32, st32, _ = timed_steps(ctx32, solver, args.steps, zeros32, stream32, torch)
            prof32 = ctx32.profile_sweeps(np.zeros(ctx32.ctrl_total), reps=5)
            extras["fp32_state"] = {"value": st32.pt_steps / (ms32 / 1e3), "unit": UNIT,
                                    "ms_per_step": ms32 / args.steps, "dtype": "f32 state, f64 reductions",
                                    "sweep_launch": ctx32.sweep_config(),
                                    "sweeps_ms": {"forward": prof32["forward_ms"],
                                                  "adjoint": prof32["adjoint_ms"],
                                                  "eval": prof32["eval_ms"]}}
            h64 = time_to_analysis(ctx, solver, truth[0], wl.max_outer, torch, stream, zeros)
            h32 = time_to_analysis(ctx32, solver, truth[0], wl.max_outer, torch, stream32, zeros32)
            target = 1.01 * h64[-1][1]
            t64 = next(t for t, r, _ in h64 if r <= target)
            t32 = next((t for t, r, _ in h32 if r <= target), None)
            extras["time_to_analysis"] = {
                "rmse_h_background": rmse_h(inp["x_b0"], truth[0]),
                "rmse_h_fp64_final": h64[-1][1], "rmse_h_fp32_final": h32[-1][1],
                "target_rmse_h": target, "fp64_s": t64, "fp32_s": t32,
                "speedup": (t64 / t32) if t32 else None,
                "outer_fp64": len(h64), "outer_fp32": len(h32)}
            ctx32.destroy()
            # Gauss-Newton local solver (Algorithms 6-7) on the FP64 path: one
            # outer step timed like the L-BFGS step, and its time to the same
            # analysis RMSE target
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
            extras["gauss_newton"] = {
                "settings": {"gn_iters": 3, "cg_iters": 10, "cg_tol": 1e-6},
                "value": st_gn.pt_steps / (ms_gn / 1e3), "unit": UNIT, "ms_per_step": ms_gn / args.steps,
                "pt_steps": "evaluations (forward + adjoint) and Gauss-Newton products (tangent-linear + "
                            "adjoint) per subdomain",
                "rmse_h_final": hgn[-1][1], "s_to_target": tgn, "outer": len(hgn),
                "speedup_vs_lbfgs_fp64": (t64 / tgn) if tgn else None}

        cpu = None
        if not args.no_cpu_baseline and world == 1:
            cpu = cpu_oracle_baseline(wl, inp)

        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if prec == 0 else "f32", "data": "synthetic",
            "config": {"workload": wl_desc(wl), "precision": "fp64" if prec == 0 else "fp32-state",
                       "step": "one DD-4DVar outer iteration from the start point (20 batched L-BFGS "
                               "iterations over all 64 subdomains + Exchange)",
                       "sweep_launch": ctx.sweep_config(),
                       "pt_steps_per_eval": pts_eval, "evals_per_step": stats.evals / args.steps,
                       "l2": "inputs larger than L2: FP64 trajectories + overlap targets "
                             f"{2 * 8 * ctx.traj_total / 1e6:.0f} MB",
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks,
            "gpu_launches": int(launches), **extras,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    ctx.destroy()
    return 0


if __name__ == "__main__":
    sys.exit(main())
