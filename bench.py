#!/usr/bin/env python3
"""Benchmark of the one-shot Parareal pass (one design iteration of Algorithm 3).

Workload (one "step"): 128x128 bilinear grid (16 641 nodes, 13 Dirichlet), Nt = 1024 fine
backward-Euler steps in N_tau = 32 slices (M = 32), SIMP k = 1e-3 + (1 - 1e-3) rho^3, unit
capacity and source, power-mean exponent p = 8; design rho ~ U(0.2, 0.8) seed 0 for the warm
start, the timed design clip(rho + U(-0.01, 0.01), 0, 1) seed 1000.  One step = assemble (a1)
+ F_pri of all slices (a2) + G_pri (a3) + forward correction (a4) + F_adj (a5) + G_adj (a3) +
reverse correction with the fused sensitivity sums (a4/a6), FP32 CG with FP64 refinement.

Metric: fine DOF*steps/s = 2 N_free Nt / t_pass (primal and adjoint), and ms per one-shot
design iteration; the comparator is sequential FP64 GPU time stepping of the same design
(chained F_pri then F_adj on one cluster, FP64 CG).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference] [--precision fp64]
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

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads as W  # noqa: E402

WORKLOAD = "oneshot128"
METRIC = "fine DOF*steps/s of the one-shot Parareal pass (ms per design iteration vs sequential FP64 GPU)"
UNIT = "DOF*steps/s"


def problem_arrays(name=WORKLOAD):
    w = W.workload(name)
    n = w["n"]
    h = w["h"]
    rho_old = W.rho_uniform(n, n, 0, 0.2, 0.8)
    rho = W.rho_warm_perturb(rho_old, seed=1000, amp=0.01)
    sink = W.dirichlet_left_centre(n, n, h)
    return w, rho_old, rho, sink


def slowest_rank_ms(ms: float, device) -> float:
    """Max over all ranks of the per-rank step time (every rank receives it).  With one process,
    or without an initialised process group, returns ms unchanged."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return ms
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank_step: float, world: int, ms: float) -> float:
    """Whole-job throughput: the units all replicas processed per step over the slowest rank's time."""
    return world * units_per_rank_step / (ms * 1e-3)


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi clock / throttle sampling in the background during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        # the raw samples (the JSON line carries their summary); PTG_CLOCKS_DIR picks the folder
        self.path = os.path.join(os.environ.get("PTG_CLOCKS_DIR", tempfile.gettempdir()), f"clocks_gpu{gpu_index}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.f.close()

    def summary(self) -> dict:
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax, "samples": len(sm),
                "reasons": sorted(reasons)}


# ---------------------------------------------------------------------------- GPU arm

def run_gpu(args):
    import torch
    import torch.distributed as dist

    from paper_2411_19030_gb300 import Operator, PassBuffers, SolveConfig, oneshot_pass, sequential_pass
    from paper_2411_19030_gb300.build import build_library

    rank, world, local = dist_env()
    if world > 1 and not dist.is_initialized():
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    if rank == 0:
        build_library()
    if world > 1:
        dist.barrier()
    w, rho_old_np, rho_np, sink = problem_arrays()
    n, Nt, Ntau, dt, p = w["n"], w["Nt"], w["Ntau"], w["dt"], w["p"]
    N_free = (n + 1) ** 2 - int(sink.sum())
    solve = SolveConfig(args.precision, rtol=args.rtol, inner_rtol=1e-4, cg_iters_max=2000, refine_max=8,
                        twolevel=args.twolevel, smooth_steps=args.smooth, local_steps=args.local, initial_guess=args.initial_guess,
                        fine_stream=args.fine_stream, coarse_stream=args.coarse_stream)
    op = Operator(n, n, w["h"], w["material"], Nt, Ntau, dt, p, sink, solve=solve, device=local)
    seq_op = Operator(n, n, w["h"], w["material"], Nt, Ntau, dt, p, sink,
                      solve=SolveConfig("fp64", rtol=1e-13, cg_iters_max=4000, refine_max=8), device=local)
    buf = PassBuffers(op)
    rho_old = torch.tensor(rho_old_np, dtype=torch.float64, device=device)
    rho = torch.tensor(rho_np, dtype=torch.float64, device=device)
    stream = torch.cuda.current_stream(device)

    # warm start: the exact sequential coarse states of rho_old (sequential FP64 pass, untimed)
    seq_op.assemble(rho_old)
    sequential_pass(seq_op, buf)
    torch.cuda.synchronize()
    flush = torch.empty(int(256e6) // 4, dtype=torch.float32, device=device)   # > L2 (129 MiB)

    kinds = ["assemble", "fine_primal", "coarse_primal", "correct_primal", "fine_adjoint", "coarse_adjoint",
             "correct_adjoint"]

    overlap = args.overlap and op.can_overlap_adjoint_coarse()
    side, hi = op.side_stream(), op.sweep_stream()
    split = buf.split_parts() if overlap else None

    def timed_step(ev):
        """One one-shot design iteration with an event pair around every ABI call.  With the
        overlap (the library default for this workload) the adjoint coarse propagators run as
        their two Theta-free parts on a second stream beside the forward correction sweep, and
        the main stream only combines them once Theta is known; ev[8], ev[9] bracket the parts."""
        from paper_2411_19030_gb300 import PTG_ADJOINT, PTG_PRIMAL
        e = ev
        e[0].record(stream)
        op.assemble(rho)
        buf.U_T_new[0].copy_(buf.U_T[0])
        buf.U_th_new[0].copy_(buf.U_th[0])
        e[1].record(stream)
        op.fine_propagate_slices(buf.U_T, buf.U_th, buf.F_T, buf.F_th, T_hist=buf.T_hist)
        e[2].record(stream)
        op.coarse_sweep(PTG_PRIMAL, buf.U_T, buf.U_th, buf.G_T, buf.G_th)
        e[3].record(stream)
        Theta = buf.U_th_new[Ntau:Ntau + 1]
        if overlap:
            # as paper_2411_19030_gb300.api.oneshot_pass with the overlap: the forward sweep on a
            # high-priority stream, the two parts of G_adj beside it
            hi.wait_event(e[3])
            op.parareal_correct(PTG_PRIMAL, buf.F_T, buf.F_th, buf.G_T, buf.G_th, buf.U_T_new, buf.U_th_new,
                                T_hist=buf.T_hist, stream=hi)
            e[4].record(hi)
            side.wait_event(e[3])
            e[8].record(side)
            op.coarse_adjoint_split(buf.V_l, buf.V_g, buf.T_hist, *split, stream=side)
            e[9].record(side)
            stream.wait_event(e[4])
            op.adjoint_sweep(buf.T_hist, Theta, buf.V_l, buf.V_g, buf.F_l, buf.F_g)
            e[5].record(stream)
            stream.wait_event(e[9])
            op.coarse_adjoint_combine(Theta, *split, buf.G_l, buf.G_g)
        else:
            op.parareal_correct(PTG_PRIMAL, buf.F_T, buf.F_th, buf.G_T, buf.G_th, buf.U_T_new, buf.U_th_new,
                                T_hist=buf.T_hist)
            e[4].record(stream)
            op.adjoint_sweep(buf.T_hist, Theta, buf.V_l, buf.V_g, buf.F_l, buf.F_g)
            e[5].record(stream)
            op.coarse_sweep(PTG_ADJOINT, buf.V_l, buf.V_g, buf.G_l, buf.G_g, T_hist=buf.T_hist, Theta=Theta)
        e[6].record(stream)
        op.parareal_correct(PTG_ADJOINT, buf.F_l, buf.F_g, buf.G_l, buf.G_g, buf.V_l_new, buf.V_g_new,
                            T_hist=buf.T_hist, Theta=Theta)
        e[7].record(stream)

    def new_events():
        return [torch.cuda.Event(enable_timing=True) for _ in range(10)]

    for _ in range(args.warmup):
        flush.fill_(1.0)
        timed_step(new_events())
    torch.cuda.synchronize()
    op.reset_stats()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    evs = []
    with ClockSampler(local) as clk:
        t0 = time.perf_counter()
        for _ in range(args.steps):
            flush.fill_(1.0)                    # L2 flushed between steps (outside the events)
            ev = new_events()
            timed_step(ev)
            evs.append(ev)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
    if world > 1:
        dist.barrier()
    per_kind = np.zeros(len(kinds))
    step_ms = []
    side_ms = []
    for ev in evs:
        d = [ev[i].elapsed_time(ev[i + 1]) for i in range(7)]
        per_kind += np.array(d)
        step_ms.append(ev[0].elapsed_time(ev[7]))
        if overlap:
            side_ms.append(ev[8].elapsed_time(ev[9]))
    ms = float(np.sum(step_ms)) / args.steps
    stats = op.stats()
    ms = slowest_rank_ms(ms, device)
    dof_steps = 2.0 * N_free * Nt
    value = job_throughput(dof_steps, world, ms)
    kind_ms = {k: float(v / args.steps) for k, v in zip(kinds, per_kind)}
    if overlap:
        # the adjoint coarse kind's solves ran on the side stream; the main stream only waited for
        # them and combined the parts (the time it shows for that kind)
        kind_ms["coarse_adjoint_combine_main"] = kind_ms.pop("coarse_adjoint")
        kind_ms["coarse_adjoint"] = float(np.mean(side_ms))

    if args.extras:
        # end to end through the public API with host buffers: H2D of rho, D2H of Theta and grad
        rho_host = torch.from_numpy(rho_np).pin_memory()
        out_host = torch.empty(1 + n * n, dtype=torch.float64).pin_memory()
        e2e_ms = []
        for _ in range(max(2, min(args.steps, 5))):
            flush.fill_(1.0)
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            rho.copy_(rho_host, non_blocking=True)
            op.assemble(rho)
            Theta, grad = oneshot_pass(op, buf)
            out_host[:1].copy_(Theta, non_blocking=True)
            out_host[1:].copy_(grad, non_blocking=True)
            b.record(stream)
            b.synchronize()
            e2e_ms.append(a.elapsed_time(b))
        e2e = float(np.mean(e2e_ms))

        # comparator: sequential FP64 GPU time stepping of the same design, one timed pass each:
        # at the one-shot's solver tolerance (the headline ratio), at rtol 1e-13 (the accuracy
        # reference below), and at the one-shot's tolerance with every CG started from the last
        # state instead of the extrapolated one (the plain scheme)
        def time_sequential(sop):
            sbuf = PassBuffers(sop)
            sop.assemble(rho)
            sequential_pass(sop, sbuf)             # untimed: plan selection and first launches
            sop.reset_stats()
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            Th, gr = sequential_pass(sop, sbuf)
            b.record(stream)
            b.synchronize()
            st = sop.stats()
            return a.elapsed_time(b), Th.clone(), gr.clone(), st

        def seq_solve(**kw):
            return SolveConfig("fp64", cg_iters_max=4000, refine_max=8, **kw)
        tight_ms, Theta_seq, grad_seq, tight_stats = time_sequential(seq_op)
        seq_alt = {}
        for key, cfg in (("tol", seq_solve(rtol=args.rtol)), ("plain", seq_solve(rtol=args.rtol, initial_guess=1))):
            sop = Operator(n, n, w["h"], w["material"], Nt, Ntau, dt, p, sink, solve=cfg, device=local)
            seq_alt[key] = time_sequential(sop)
            del sop
        seq_ms, _, _, seq_stats = seq_alt["tol"]
        # accuracy of the one-shot estimate and of the mixed arithmetic against sequential FP64
        Theta_os = float(buf.U_th_new[Ntau].item())
        g_os = buf.V_g_new[0]
        err_theta = abs(Theta_os - float(Theta_seq.item())) / abs(float(Theta_seq.item()))
        err_grad = float(torch.linalg.norm(g_os - grad_seq) / torch.linalg.norm(grad_seq))
        # error of the precision pattern: the same one-shot pass in FP64 (CG and all sums FP64,
        # rtol 1e-13; this path matches the CPU oracle to 1e-10 in the parity tests), untimed
        prec = {}
        fp64_arm = None
        if args.precision != "fp64":
            f64_op = Operator(n, n, w["h"], w["material"], Nt, Ntau, dt, p, sink,
                              solve=SolveConfig("fp64", rtol=1e-13, cg_iters_max=8000, refine_max=8), device=local)
            f64_buf = PassBuffers(f64_op)
            for a_, b_ in ((f64_buf.U_T, buf.U_T), (f64_buf.U_th, buf.U_th), (f64_buf.V_l, buf.V_l), (f64_buf.V_g, buf.V_g)):
                a_.copy_(b_)
            # timed like the main steps: the FP64 half of the configuration (FP64 vs FP32 CG + FP64
            # refinement); its comparator is sequential FP64 stepping at the same rtol 1e-13
            f64_ms = []
            for i in range(args.warmup + args.steps):
                flush.fill_(1.0)
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                f64_op.assemble(rho)
                Th64, g64 = oneshot_pass(f64_op, f64_buf)
                b.record(stream)
                b.synchronize()
                if i >= args.warmup:
                    f64_ms.append(a.elapsed_time(b))
            f64_mean = slowest_rank_ms(float(np.mean(f64_ms)), device)
            f64_st = f64_op.stats()
            fp64_arm = {"what": "the same one-shot pass with every CG and sum in FP64 (rtol 1e-13), timed like the "
                                "main steps", "ms_per_step": f64_mean, "value": job_throughput(dof_steps, world, f64_mean),
                        "unit": UNIT, "sequential_fp64_rtol_1e-13_ms": tight_ms,
                        "speedup_vs_sequential_fp64_same_rtol": tight_ms / f64_mean,
                        "mixed_over_fp64_speedup": f64_mean / ms,
                        "cg_per_solve": {k: round(v["cg_iters"] / max(1, v["solves"]), 2)
                                         for k, v in f64_st["by_kind"].items() if v["solves"]}}

            def relmax(a, b):
                return float((a - b).abs().max() / b.abs().max())
            f64_T = f64_buf.T_hist
            prec = {"T_hist_rel_max": relmax(buf.T_hist, f64_T),
                    "Theta_rel": abs(Theta_os - float(Th64.item())) / abs(float(Th64.item())),
                    "grad_rel_max": relmax(g_os, g64),
                    "targets": {"temperature": 1e-6, "sensitivity": 1e-5}}

        # the other mixed variant (every CG in FP32 when the headline keeps the coarse solves in
        # FP64, and the reverse), timed like the main steps, with its error against FP64
        variant = None
        if args.precision != "fp64":
            vname = "fp32_refine_all" if args.precision == "fp32_refine" else "fp32_refine"
            v_op = Operator(n, n, w["h"], w["material"], Nt, Ntau, dt, p, sink,
                            solve=SolveConfig(vname, rtol=args.rtol, inner_rtol=1e-4, cg_iters_max=2000,
                                              refine_max=8, twolevel=args.twolevel, smooth_steps=args.smooth, local_steps=args.local, initial_guess=args.initial_guess), device=local)
            v_buf = PassBuffers(v_op)
            for a_, b_ in ((v_buf.U_T, buf.U_T), (v_buf.U_th, buf.U_th), (v_buf.V_l, buf.V_l),
                           (v_buf.V_g, buf.V_g)):
                a_.copy_(b_)
            v_ms = []
            for i in range(args.warmup + args.steps):
                flush.fill_(1.0)
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                v_op.assemble(rho)
                Thv, gv = oneshot_pass(v_op, v_buf)
                b.record(stream)
                b.synchronize()
                if i >= args.warmup:
                    v_ms.append(a.elapsed_time(b))
            vm = slowest_rank_ms(float(np.mean(v_ms)), device)
            variant = {"precision": vname, "ms_per_step": vm, "value": job_throughput(dof_steps, world, vm),
                       "unit": UNIT, "speedup_vs_sequential_fp64": seq_ms / vm,
                       "T_hist_rel_max": relmax(v_buf.T_hist, f64_T), "grad_rel_max": relmax(gv, g64)}
            del v_buf, f64_buf

        # Sec. 7.3 future work: the same pass with the coarse propagators on the 2h mesh, timed
        # like the main steps, with the error of its one-shot estimate against the sequential result
        c_op = Operator(n, n, w["h"], w["material"], Nt, Ntau, dt, p, sink,
                        solve=SolveConfig(args.precision, rtol=args.rtol, inner_rtol=1e-4, cg_iters_max=2000,
                                          refine_max=8, twolevel=args.twolevel, smooth_steps=args.smooth, local_steps=args.local, initial_guess=args.initial_guess,
                                          coarse_mesh=True), device=local)
        c_buf = PassBuffers(c_op)
        for a_, b_ in ((c_buf.U_T, buf.U_T), (c_buf.U_th, buf.U_th), (c_buf.V_l, buf.V_l), (c_buf.V_g, buf.V_g)):
            a_.copy_(b_)
        c_ms = []
        for i in range(args.warmup + args.steps):
            flush.fill_(1.0)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            c_op.assemble(rho)
            Thc, gc = oneshot_pass(c_op, c_buf)
            b.record(stream)
            b.synchronize()
            if i >= args.warmup:
                c_ms.append(a.elapsed_time(b))
        cm_ms = slowest_rank_ms(float(np.mean(c_ms)), device)
        cst = c_op.stats()
        coarse_mesh = {"what": "Sec. 7.3 future work: G_pri and G_adj on the 2h mesh (64x64 elements)",
                       "ms_per_step": cm_ms, "value": job_throughput(dof_steps, world, cm_ms), "unit": UNIT,
                       "speedup_vs_sequential_fp64": seq_ms / cm_ms, "status": cst["status"],
                       "Theta_rel_vs_sequential": abs(float(Thc.item()) - float(Theta_seq.item()))
                       / abs(float(Theta_seq.item())),
                       "grad_rel_l2_vs_sequential": float(torch.linalg.norm(gc - grad_seq) / torch.linalg.norm(grad_seq)),
                       "cg_per_solve": {k: round(v["cg_iters"] / max(1, v["solves"]), 2)
                                        for k, v in cst["by_kind"].items() if v["solves"]}}
        del c_buf, c_op

        # Sec. 7.3 bottleneck probe: the same pass with the coarse propagators identically zero
        # (G_pri = G_adj = 0, the corrections copy F), timed like the main steps
        g0_ms = []
        for i in range(args.warmup + args.steps):
            flush.fill_(1.0)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            op.assemble(rho)
            oneshot_pass(op, buf, plt=True)
            b.record(stream)
            b.synchronize()
            if i >= args.warmup:
                g0_ms.append(a.elapsed_time(b))
        g0 = slowest_rank_ms(float(np.mean(g0_ms)), device)
        probe = {"what": "Sec. 7.3: the one-shot pass with G_pri = G_adj = 0 (PLT-style corrections) at N_tau = 32",
                 "oneshot_ms": ms, "g_zero_ms": g0, "sequential_fp64_ms": seq_ms,
                 "speedup_oneshot": seq_ms / ms, "speedup_g_zero": seq_ms / g0,
                 "paper_context": "MATLAB on 32 CPU threads: 3.81x (one-shot) vs 10.8x (G = 0) over its sequential run"}
    else:
        e2e = seq_ms = None
        seq_stats, prec, probe, variant, coarse_mesh, fp64_arm = {}, {}, None, None, None, None
        err_theta = err_grad = None

    roof = roofline(kind_ms, stats, N_free, args.steps, args.precision)
    streaming = streaming_256(args, flush, stream, device) if (args.extras and args.c3) else None
    batch48 = None
    if args.extras and args.c4 and world == 1:
        bl = batch48_line(args, steps=3, autotune_plans=False)
        batch48 = {k: bl[k] for k in ("ms_per_batched_pass", "design_by_design_ms", "batching_speedup", "value",
                                      "unit", "steps", "designs_on_own_path", "status")}
        batch48["workload"] = bl["config"]["workload"]
    loop512 = None
    if args.extras and args.c5 and world == 1:
        ll = loop_line(args, 3)
        loop512 = {"what": "Alg. 3 at 512x512 (Nt = 4096, 128 slices), 3 design iterations (1 sequential, 2 one-shot); "
                           "the comparator is sequential FP64 time stepping of the last design",
                   "workload": ll["config"]["workload"], "ms_per_oneshot_iteration": ll["value"],
                   "iteration_ms": ll["history"]["ms"], "sequential_fp64_ms": ll["sequential_fp64_ms_last_design"],
                   "speedup_vs_sequential_fp64": ll["speedup_last_iteration_vs_sequential_fp64"],
                   "Theta_estimate": ll["final"]["Theta_estimate"],
                   "Theta_true_fp64_sequential": ll["final"]["Theta_true_fp64_sequential"]}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f32+f64",
        "data": "synthetic",
        "config": {"workload": f"{WORKLOAD}: 128x128 grid, Nt=1024, Ntau=32 (M=32), p=8, SIMP k, warm start from "
                               "the sequential coarse states of a design 1% away",
                   "overlap_adjoint_coarse": overlap,
                   "precision": args.precision, "rtol": args.rtol, "twolevel": args.twolevel, "smooth_steps": args.smooth, "local_steps": args.local, "initial_guess": args.initial_guess, "fine_stream": args.fine_stream, "coarse_stream": args.coarse_stream, "l2": "flushed between steps (256 MB write)",
                   "parallelism": f"replicas x{world}" if world > 1 else "1 GPU",
                   "wall_s": wall},
        "per_kernel_ms": kind_ms,
        # the metric per F phase: N_free * Nt fine DOF-steps in the fine primal and in the fine
        # adjoint propagator alone, beside the whole pass (2 N_free Nt per pass)
        "phase_dof_steps_per_s": {
            k: N_free * Nt / (max(kind_ms.get(k, 0.0), 1e-9) * 1e-3) for k in ("fine_primal", "fine_adjoint")},
        "cg": {"solves": stats["solves"], "cg_iters": stats["cg_iters"], "refinements": stats["refinements"],
               "mean_cg_per_solve": stats["cg_iters"] / max(1, stats["solves"]),
               "by_kind": {k: {"cg_per_solve": v["cg_iters"] / max(1, v["solves"]),
                               "refine_per_solve": v["refinements"] / max(1, v["solves"])}
                           for k, v in stats["by_kind"].items() if v["solves"]}},
        "comparator_sequential_fp64": None if seq_ms is None else {
            "what": f"sequential FP64 time stepping (chained F_pri, F_adj) at rtol {args.rtol:g}, each CG started "
                    "from the extrapolation through the last 4 states (the library default)",
            "ms": seq_ms, "value": dof_steps / (seq_ms * 1e-3), "unit": UNIT, "speedup_of_oneshot": seq_ms / ms,
            "cg_iters": seq_stats["cg_iters"], "solves": seq_stats["solves"],
            "variants": {
                "rtol_1e-13": {"ms": tight_ms, "speedup_of_oneshot": tight_ms / ms, "cg_iters": tight_stats["cg_iters"]},
                "plain_start": {"what": "every CG started from the last state", "ms": seq_alt["plain"][0],
                                "speedup_of_oneshot": seq_alt["plain"][0] / ms,
                                "cg_iters": seq_alt["plain"][3]["cg_iters"]}}},
        "accuracy_vs_sequential_fp64": {"Theta_rel": err_theta, "grad_rel_l2": err_grad,
                                        "note": "one-shot estimate (warm start from a design 1% away) vs the exact "
                                                "sequential result of the current design"},
        "accuracy_mixed_vs_fp64_oneshot": prec,
        "bottleneck_probe": probe,
        "coarse_mesh_variant": coarse_mesh,
        "precision_variant": variant,
        "fp64_oneshot": fp64_arm,
        "streaming_256": streaming,
        "batch48": batch48,
        "loop512": loop512,
        "e2e": None if e2e is None else {"value": world * dof_steps / (e2e * 1e-3), "unit": UNIT, "ms": e2e,
                                         "h2d_bytes_per_step": n * n * 8, "d2h_bytes_per_step": (1 + n * n) * 8},
        # per pass: assembly 3 kernels, the two-level set-up 4 (+ 5 for the three-level one), and
        # the pass: F_pri, G_pri, the two sweeps, F_adj and G_adj (overlapped: its two parts and
        # the combination)
        "gpu_launches": (3 + (4 if args.twolevel != "none" else 0) + (5 if args.twolevel == "threelevel" else 0)
                         + (8 if overlap else 6)) * args.steps,
        "roofline": roof,
        "clocks": clk.summary(),
    }
    if rank == 0:
        if args.cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(args.cpu_seconds)
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


# DRAM bytes per launch (read + write) of the 128x128 pass in the default precision, from one
# ncu capture (profiles/).  They hold only for that workload and precision, and only for the
# kernel source they were taken from: the hash of the stepper sources at capture time is stored
# beside them.  Any other workload, precision or source hash reports traffic as null.
NCU_TRAFFIC = {
    "captured": "2026-12-03",
    "sources_sha16": "a6f7f5ec6bb57ab9",
    "workload": WORKLOAD,
    "precision": "fp32_refine",
    # the adjoint coarse propagator runs as its two Theta-free parts (two launches per pass)
    "bytes": {"fine_primal": 8.002304e6 + 108.280064e6, "coarse_primal": 7.368448e6 + 256.0,
              "correct_primal": 11.627264e6 + 768.0, "fine_adjoint": 149.358848e6 + 2.136320e6,
              "coarse_adjoint": (15.459840e6 + 0.0) + (7.042304e6 + 512.0),
              "correct_adjoint": 24.212224e6 + 0.0},
}
STEPPER_SOURCES = ("stepper.cuh", "comm.cuh", "ptg_device.cuh", "stepper_inst.cu", "stepper_launch.cuh", "plan.cu")


def stepper_sources_sha16() -> str:
    import hashlib
    hsh = hashlib.sha256()
    for name in STEPPER_SOURCES:
        with open(os.path.join(ROOT, "paper_2411_19030_gb300", "csrc", name), "rb") as f:
            hsh.update(f.read())
    return hsh.hexdigest()[:16]


def ncu_traffic(kind: str, workload: str = WORKLOAD, precision: str = "fp32_refine"):
    """(bytes per launch or None, provenance) of the stored ncu DRAM figure of a kernel."""
    if workload != NCU_TRAFFIC["workload"] or precision != NCU_TRAFFIC["precision"]:
        return None, (f"no ncu capture of this workload and precision ({workload}, {precision}); the stored one "
                      f"is of {NCU_TRAFFIC['workload']}, {NCU_TRAFFIC['precision']}")
    sha = stepper_sources_sha16()
    if NCU_TRAFFIC["sources_sha16"] != sha or kind not in NCU_TRAFFIC["bytes"]:
        return None, f"no ncu capture of the current stepper sources ({sha})"
    return NCU_TRAFFIC["bytes"][kind], f"ncu capture of {NCU_TRAFFIC['captured']}, stepper sources {sha}"


# FP64 peak of the chip (nominal, 1.25 TFLOP/s; MEASURED_PEAKS.json holds no FP64 figure) and the
# FLOPs of one FP64 CG iteration per unknown: the 9-point stencil (9 FMA), the p, q, d, r
# updates (4 FMA), three dot products (3 FMA) and the preconditioned residual (1 FMA) = 17 FMA;
# one FP64 residual evaluation per refinement sweep and per solve: stencil + subtraction + dot.
FP64_PEAK_TFLOPS = 1.25
FLOPS_PER_CG_ITER = 34.0
FLOPS_PER_RESIDUAL = 21.0
KIND_PRECISION = {"fp64": {k: "f64" for k in ("fine_primal", "coarse_primal", "correct_primal", "fine_adjoint",
                                              "coarse_adjoint", "correct_adjoint")},
                  "fp32_refine_all": {k: "f32" for k in ("fine_primal", "coarse_primal", "correct_primal",
                                                         "fine_adjoint", "coarse_adjoint", "correct_adjoint")},
                  "fp32_refine": {"fine_primal": "f32", "fine_adjoint": "f32", "coarse_primal": "f64",
                                  "correct_primal": "f64", "coarse_adjoint": "f64", "correct_adjoint": "f64"}}
ADJOINT_KINDS = ("fine_adjoint", "coarse_adjoint", "correct_adjoint")


def hbm_peak():
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    if "hbm_gbs" in peaks:
        return float(peaks["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs, a STREAM-style copy)"
    return 6800.0, "fallback 6800 GB/s (no MEASURED_PEAKS.json)"


def algorithmic_bytes(kind: str, st: dict, N_free: int, launches: int) -> float:
    """Algorithmic HBM bytes of one launch of a stepper kind, counted per free DOF and solve as
    if every CG vector streamed from memory: 16 B per solve (the previous state read, the new
    state written, FP64), 36 B per CG iteration (p, x, r, Ap and the coefficients read; Ap, x,
    r, p written), 28 B per FP64 refinement sweep (T, b and the coefficients read; r written),
    and 8 B more per adjoint solve (the T_j read shared by the source and the sensitivity
    sum).  The solver counters give the iterations and sweeps; `launches` is the number of
    launches they cover."""
    per_dof = (16.0 + (8.0 if kind in ADJOINT_KINDS else 0.0)) * st["solves"] + 36.0 * st["cg_iters"] \
        + 28.0 * st["refinements"]
    return N_free * per_dof / max(1, launches)


def roofline(kind_ms: dict, stats: dict, N_free: int, launches: int, precision: str,
             workload: str = WORKLOAD) -> dict:
    """Roofline entry of the dominant kernel (largest share of the step) against the measured
    HBM copy bandwidth, with the algorithmic bytes of algorithmic_bytes(); beside it every
    stepper kernel's figure, and for an FP64-CG kernel its algorithmic FP64 FLOP rate against
    the nominal FP64 peak (context: the chip runs FP64 at 1/58 of its FP32 rate)."""
    hbm, source = hbm_peak()
    per = {}
    for k, ms in kind_ms.items():
        st = stats["by_kind"].get(k)
        if not st or not st["solves"]:
            continue
        b = algorithmic_bytes(k, st, N_free, launches)
        gbs = b / (ms * 1e-3) / 1e9
        per[k] = {"ms": ms, "algorithmic_bytes": b, "achieved_gbs": gbs, "frac": gbs / hbm,
                  "solves": st["solves"] / max(1, launches), "cg_per_solve": st["cg_iters"] / max(1, st["solves"]),
                  "refine_per_solve": st["refinements"] / max(1, st["solves"])}
    dom = max(per, key=lambda k: per[k]["ms"])
    d = per[dom]
    traffic, tsrc = ncu_traffic(dom, workload, precision)
    out = {"kernel": dom, "bound": "hbm", "achieved": d["achieved_gbs"], "peak": hbm, "unit": "GB/s",
           "frac": d["frac"], "traffic": traffic, "traffic_source": tsrc, "peak_source": source,
           "algorithmic_bytes_per_launch": d["algorithmic_bytes"],
           "bytes_rule": "N_free x (16 B per solve (+8 adjoint) + 36 B per CG iteration + 28 B per FP64 refinement "
                         "sweep), from the kernel's own solver counters",
           "per_kernel": per}
    if KIND_PRECISION[precision][dom] == "f64":
        st = stats["by_kind"][dom]
        flops = N_free * (FLOPS_PER_CG_ITER * st["cg_iters"] + FLOPS_PER_RESIDUAL * (st["refinements"] + st["solves"]))
        flops /= max(1, launches)
        tf = flops / (kind_ms[dom] * 1e-3) / 1e12
        out["fp64_alu"] = {"achieved_tflops": tf, "peak_tflops": FP64_PEAK_TFLOPS, "frac": tf / FP64_PEAK_TFLOPS,
                           "peak_source": "nominal FP64 peak of the chip (no measured FP64 peak)"}
    out["note"] = ("the CG vectors of a system stay on chip, so the bytes are what a streaming CG would move; the "
                   "correction sweeps are sequential (one system on one 16-CTA cluster at a time) and bound by the "
                   "latency of their cluster barriers and by the FP64 pipes of 16 SMs, not by HBM")
    return out


def streaming_256(args, flush, stream, device, name="diff256") -> dict:
    """The one-shot pass on the 256x256 workload (Nt = 2048 in 64 slices, rho ~ U(0, 1) seed 1, the
    timed design 1% away from the warm start's, seed 1000), the grid size at which the history
    (1.08 GB) and a slice batch no longer fit in L2: per-kernel CUDA-event times and each stepper
    kernel's algorithmic bandwidth against the measured HBM copy bandwidth.  Warm start from the
    sequential FP64 coarse states of the nearby design (untimed).  name = "loop512" takes the
    512x512 sizes (Nt = 4096 in 128 slices) with the same design recipe."""
    import torch

    from paper_2411_19030_gb300 import Operator, PassBuffers, SolveConfig, sequential_pass
    from paper_2411_19030_gb300 import PTG_ADJOINT, PTG_PRIMAL

    w = W.workload(name)
    n, Nt, Ntau, dt, p = w["n"], w["Nt"], w["Ntau"], w["dt"], w["p"]
    sink = W.dirichlet_left_centre(n, n, w["h"])
    N_free = (n + 1) ** 2 - int(sink.sum())
    rho_old_np = W.rho_uniform(n, n, 1, 0.0, 1.0)
    rho_np = W.rho_warm_perturb(rho_old_np, seed=1000, amp=0.01)
    solve = SolveConfig(args.precision, rtol=args.rtol, inner_rtol=1e-4, cg_iters_max=4000, refine_max=8,
                        twolevel=args.twolevel, smooth_steps=args.smooth, local_steps=args.local,
                        initial_guess=args.initial_guess, fine_stream=args.fine_stream, coarse_stream=args.coarse_stream)
    op = Operator(n, n, w["h"], w["material"], Nt, Ntau, dt, p, sink, solve=solve, device=device.index)
    wop = Operator(n, n, w["h"], w["material"], Nt, Ntau, dt, p, sink,
                   solve=SolveConfig("fp64", rtol=1e-12, cg_iters_max=8000, refine_max=8), device=device.index)
    buf = PassBuffers(op)
    rho_old = torch.tensor(rho_old_np, dtype=torch.float64, device=device)
    rho = torch.tensor(rho_np, dtype=torch.float64, device=device)
    wop.assemble(rho_old)
    sequential_pass(wop, buf)
    torch.cuda.synchronize()
    del wop
    kinds = ["assemble", "fine_primal", "coarse_primal", "correct_primal", "fine_adjoint", "coarse_adjoint",
             "correct_adjoint"]

    def step(e):
        e[0].record(stream)
        op.assemble(rho)
        e[1].record(stream)
        op.fine_propagate_slices(buf.U_T, buf.U_th, buf.F_T, buf.F_th, T_hist=buf.T_hist)
        e[2].record(stream)
        op.coarse_sweep(PTG_PRIMAL, buf.U_T, buf.U_th, buf.G_T, buf.G_th)
        e[3].record(stream)
        buf.U_T_new[0].copy_(buf.U_T[0])
        buf.U_th_new[0].copy_(buf.U_th[0])
        op.parareal_correct(PTG_PRIMAL, buf.F_T, buf.F_th, buf.G_T, buf.G_th, buf.U_T_new, buf.U_th_new,
                            T_hist=buf.T_hist)
        e[4].record(stream)
        Theta = buf.U_th_new[Ntau:Ntau + 1]
        op.adjoint_sweep(buf.T_hist, Theta, buf.V_l, buf.V_g, buf.F_l, buf.F_g)
        e[5].record(stream)
        op.coarse_sweep(PTG_ADJOINT, buf.V_l, buf.V_g, buf.G_l, buf.G_g, T_hist=buf.T_hist, Theta=Theta)
        e[6].record(stream)
        op.parareal_correct(PTG_ADJOINT, buf.F_l, buf.F_g, buf.G_l, buf.G_g, buf.V_l_new, buf.V_g_new,
                            T_hist=buf.T_hist, Theta=Theta)
        e[7].record(stream)

    flush.fill_(1.0)
    step([torch.cuda.Event(enable_timing=True) for _ in range(8)])      # warm-up: plans, attributes
    torch.cuda.synchronize()
    op.reset_stats()
    per = np.zeros(7)
    tot = []
    for _ in range(max(1, args.c3_steps)):
        flush.fill_(1.0)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(8)]
        step(ev)
        torch.cuda.synchronize()
        per += np.array([ev[i].elapsed_time(ev[i + 1]) for i in range(7)])
        tot.append(ev[0].elapsed_time(ev[7]))
    steps = max(1, args.c3_steps)
    kind_ms = {k: float(v / steps) for k, v in zip(kinds, per)}
    st = op.stats()
    ms = float(np.mean(tot))
    roof = roofline(kind_ms, st, N_free, steps, args.precision, name)
    out = {"workload": f"{name}: {n}x{n} grid, Nt={Nt}, Ntau={Ntau} (M={Nt // Ntau}), p={p:g}, rho ~ U(0,1) seed 1, "
                       "timed design 1% away (seed 1000), warm start from the sequential FP64 coarse states",
           "precision": args.precision, "rtol": args.rtol, "steps": steps, "ms_per_step": ms,
           "value": 2.0 * N_free * Nt / (ms * 1e-3), "unit": UNIT, "per_kernel_ms": kind_ms,
           "status": st["status"], "roofline": roof}
    del buf, op
    torch.cuda.synchronize()
    return out


def run_c3_only(args):
    import torch

    from paper_2411_19030_gb300.build import build_library
    build_library()
    device = torch.device("cuda", 0)
    torch.cuda.set_device(device)
    flush = torch.empty(int(256e6) // 4, dtype=torch.float32, device=device)
    print(json.dumps(streaming_256(args, flush, torch.cuda.current_stream(device), device, args.c3_workload)),
          flush=True)


# ---------------------------------------------------------------------------- full design loop

def run_loop(args):
    print(json.dumps(loop_line(args, args.loop)), flush=True)


def loop_line(args, iterations):
    """Alg. 3 at 512 x 512, Nt = 4096 in 128 slices (M = 32): rho(0) = a_max = 0.4 uniform, the
    paper's filter and projection (r_fil = 0.03, beta = 32, eta = 0.5, no continuation), host MMA
    (move 0.2); design iteration 1 sequential, the rest one-shot.  Reports the time of every
    design iteration and the objective history; the true objective of the final design by a
    sequential FP64 pass, outside the timed loop, whose time is the comparator for the last
    one-shot iteration (same design)."""
    import torch

    from paper_2411_19030_gb300 import Operator, SolveConfig
    from paper_2411_19030_gb300.build import build_library
    from paper_2411_19030_gb300.design import DesignMap, OneShotLoop

    build_library()
    n = args.loop_n
    w = W.workload("loop512")
    Nt, Ntau = (w["Nt"], w["Ntau"]) if n == 512 else (8 * n, n // 4)
    h = 1.0 / n
    dt = 1.0 / Nt
    sink = W.dirichlet_left_centre(n, n, h)
    a_max, r_fil, beta, eta = 0.4, 0.03, 32.0, 0.5
    op = Operator(n, n, h, w["material"], Nt, Ntau, dt, w["p"], sink,
                  solve=SolveConfig(args.precision, rtol=args.rtol, inner_rtol=1e-4, cg_iters_max=4000, refine_max=8,
                                    twolevel=args.twolevel, smooth_steps=args.smooth, local_steps=args.local, initial_guess=args.initial_guess, coarse_mesh=args.coarse_mesh,
                                    fine_stream=args.fine_stream, coarse_stream=args.coarse_stream))
    true_op = Operator(n, n, h, w["material"], Nt, Ntau, dt, w["p"], sink,
                       solve=SolveConfig("fp64", rtol=1e-12, cg_iters_max=8000, refine_max=8,
                                         initial_guess=args.initial_guess))
    design = DesignMap(n, n, h, r_fil, beta, eta)
    loop = OneShotLoop(op, design, a_max, move=0.2, true_op=true_op)
    # uniform chi with P(chi) = a_max (the filter keeps a uniform field)
    den = np.tanh(beta * (1 - eta)) + np.tanh(beta * eta)
    chi0 = np.full(n * n, eta + np.arctanh(a_max * den - np.tanh(beta * eta)) / beta)
    with ClockSampler(0) as clk:
        t0 = time.perf_counter()
        hist = loop.run(chi0, iterations, true_every=0)
        wall = time.perf_counter() - t0
    torch.cuda.synchronize()
    # the comparator on the design of the last iteration: sequential FP64 time stepping (the
    # buffers are allocated before the timed pass)
    from paper_2411_19030_gb300 import PassBuffers, sequential_pass
    tb = PassBuffers(true_op)
    true_op.assemble(loop.rho)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    Theta_true, _ = sequential_pass(true_op, tb)
    torch.cuda.synchronize()
    seq_ms = 1e3 * (time.perf_counter() - t1)
    true_final = float(Theta_true.item())
    del tb
    ms = hist["ms"]
    oneshot = ms[1:] if len(ms) > 1 else ms
    N_free = (n + 1) ** 2 - int(sink.sum())
    line = {
        "metric": "ms per one-shot design iteration (full design loop, host MMA)", "value": float(np.mean(oneshot)),
        "unit": "ms", "higher_is_better": False, "n_gpus": 1, "steps": len(ms), "warmup": 0,
        "dtype": "f64" if args.precision == "fp64" else "f32+f64", "data": "synthetic",
        "config": {"workload": f"loop{n}: {n}x{n} grid, Nt={Nt}, Ntau={Ntau}, p=8, SIMP k, a_max={a_max}, "
                               f"r_fil={r_fil}, beta={beta}, eta={eta}, MMA move 0.2",
                   "precision": args.precision, "rtol": args.rtol, "twolevel": args.twolevel, "smooth_steps": args.smooth, "local_steps": args.local, "initial_guess": args.initial_guess, "fine_stream": args.fine_stream, "coarse_stream": args.coarse_stream,
                   "coarse_propagator": "2h mesh (Sec. 7.3 future work)" if args.coarse_mesh else "h mesh"},
        "first_iteration_sequential_ms": ms[0],
        "fine_dof_steps_per_s": 2.0 * N_free * Nt / (np.mean(oneshot) * 1e-3),
        "history": {"Theta_estimate": hist["Theta"], "area_fraction": hist["volume"], "ms": ms},
        "final": {"Theta_estimate": hist["Theta"][-1], "Theta_true_fp64_sequential": true_final,
                  "area_fraction": hist["volume"][-1]},
        "sequential_fp64_ms_last_design": seq_ms,
        "speedup_last_iteration_vs_sequential_fp64": seq_ms / ms[-1],
        "wall_s": wall, "clocks": clk.summary(),
    }
    del loop, op, true_op
    torch.cuda.synchronize()
    return line


# ---------------------------------------------------------------------------- batching

def run_batch48(args):
    print(json.dumps(batch48_line(args)), flush=True)


def batch48_line(args, steps=None, autotune_plans=None):
    """The batching workload: 48 designs of uneven size (64^2 .. 256^2, Nt 512 .. 2048, 16 .. 64
    slices), warm-started from the sequential coarse states of designs 1% away, advanced
    together: each phase of the one-shot pass is one persistent launch over every design and
    slice, assembly plus pass captured in one CUDA graph and replayed.  Reports the aggregate
    fine DOF*steps/s of the batched pass, and the time of the same 48 passes run design by
    design (each with its own plans), both with CUDA events and the L2 flushed before each."""
    import torch

    from paper_2411_19030_gb300 import Operator, PassBuffers, SolveConfig, oneshot_pass, sequential_pass
    from paper_2411_19030_gb300.batch import Batch, autotune
    from paper_2411_19030_gb300.build import build_library

    build_library()
    device = torch.device("cuda", 0)
    designs = W.batch48()
    solve = SolveConfig(args.precision, rtol=args.rtol, inner_rtol=1e-4, cg_iters_max=2000, refine_max=8,
                        twolevel=args.twolevel, smooth_steps=args.smooth, initial_guess=args.initial_guess)
    mats = W.MATERIALS["simp_k"]
    ops, dof = [], 0.0
    for d in designs:
        n, h = d["n"], 1.0 / d["n"]
        sink = W.dirichlet_left_centre(n, n, h)
        ops.append(Operator(n, n, h, mats, d["Nt"], d["Ntau"], d["dt"], d["p"], sink, solve=solve))
        dof += 2.0 * ((n + 1) ** 2 - int(sink.sum())) * d["Nt"]
    batch = Batch(ops)
    dv = lambda a: torch.tensor(a, dtype=torch.float64, device=device)
    for i, d in enumerate(designs):
        batch.buffers(i)["rho"].copy_(dv(W.rho_warm_perturb(d["rho"], seed=1000 + d["index"], amp=0.01)))
    batch.assemble()
    batch.sequential_pass()
    for i, d in enumerate(designs):
        batch.buffers(i)["rho"].copy_(dv(d["rho"]))
    batch.assemble()
    tuned = autotune(batch) if (args.autotune if autotune_plans is None else autotune_plans) else None
    batch.oneshot_pass()
    batch.capture()
    flush = torch.empty(int(256e6) // 4, dtype=torch.float32, device=device)
    stream = torch.cuda.current_stream(device)
    steps = max(1, min(args.steps if steps is None else steps, 5))
    for _ in range(max(1, args.warmup)):
        batch.replay()
    torch.cuda.synchronize()
    times = []
    with ClockSampler(0) as clk:
        for _ in range(steps):
            flush.fill_(1.0)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            batch.replay()
            b.record(stream)
            b.synchronize()
            times.append(a.elapsed_time(b))
    ms = float(np.mean(times))
    status = max(op.stats()["status"] != 0 for op in ops)
    # the same 48 passes design by design (warm start copied from the batch's buffers)
    single = 0.0
    for i, op in enumerate(ops):
        bi = batch.buffers(i)
        buf = PassBuffers(op)
        for a_, k in ((buf.U_T, "U_T"), (buf.U_th, "U_theta"), (buf.V_l, "V_lam"), (buf.V_g, "V_g")):
            a_.copy_(bi[k])
        rho = bi["rho"].clone()
        for rep in range(2):
            flush.fill_(1.0)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            op.assemble(rho)
            oneshot_pass(op, buf)
            b.record(stream)
            b.synchronize()
        single += a.elapsed_time(b)
        del buf
    own = sum(batch.own_path(d) for d in range(len(ops)))
    line = {"metric": "fine DOF*steps/s of the batched one-shot pass (48 designs of uneven size)",
            "value": dof / (ms * 1e-3), "unit": UNIT, "ms_per_batched_pass": ms, "steps": steps,
            "design_by_design_ms": single, "batching_speedup": single / ms, "status": int(status),
            "designs_on_own_path": own,
            "autotuned": tuned is not None, "dtype": "f32+f64" if args.precision != "fp64" else "f64",
            "config": {"workload": "batch48: 48 designs, sides 64/96/128/192/256, (Nt, Ntau) in "
                                   "(512,16)/(1024,32)/(2048,64), rho ~ U(0.2,0.8)",
                       "precision": args.precision, "rtol": args.rtol, "twolevel": args.twolevel,
                       "initial_guess": args.initial_guess,
                       "l2": "flushed between steps (256 MB write)"},
            "clocks": clk.summary()}
    batch.close()
    del batch, ops
    torch.cuda.synchronize()
    return line


# ---------------------------------------------------------------------------- Parareal sweep

def run_sweep(args):
    """Sec. 5.2 on the GPU: k-iteration Parareal of the paper's test case for N_tau in divisors
    of 480 and k = 1..8, FP64, against sequential FP64 time stepping of the same design with the
    same solver: relative errors of Theta and of the gradient (2-norm) as defined in Sec. 5.2,
    and the speedup of the Parareal run over the sequential run (CUDA events, one warm-up run
    each).  Designs: rho = 0.3 uniform, and a near-binary branched stand-in for an optimised
    design (high contrast)."""
    import torch

    from paper_2411_19030_gb300 import Operator, PassBuffers, SolveConfig, parareal_pass, sequential_pass
    from paper_2411_19030_gb300.build import build_library

    build_library()
    n, Nt = 100, 480
    w = W.workload("paper100")
    h, dt = 1.0 / n, 1.0 / Nt
    sink = W.dirichlet_bottom_centre(n, n, h)
    qt = W.q_time_paper(Nt, dt)
    solve = SolveConfig("fp64", rtol=1e-12, cg_iters_max=8000, refine_max=8, coarse_mesh=args.coarse_mesh,
                        initial_guess=args.initial_guess)
    seq_solve = SolveConfig("fp64", rtol=1e-12, cg_iters_max=8000, refine_max=8, initial_guess=args.initial_guess)
    stream = torch.cuda.current_stream()

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        out = fn()
        b.record(stream)
        b.synchronize()
        return a.elapsed_time(b), out

    rows = []
    for dname, rho_np in (("uniform0.3", np.full(n * n, 0.3)), ("branches", W.rho_branches(n, n))):
        rho = torch.tensor(rho_np, dtype=torch.float64, device="cuda")
        ntaus = [int(v) for v in args.sweep_ntau.split(",")]
        seq_op = Operator(n, n, h, w["material"], Nt, ntaus[0], dt, w["p"], sink, q_time=qt, solve=seq_solve)
        seq_op.assemble(rho)
        seq_buf = PassBuffers(seq_op)
        t_seq, (Th_s, g_s) = timed(lambda: sequential_pass(seq_op, seq_buf))
        Th_s, g_s = float(Th_s.item()), g_s.clone()
        del seq_buf, seq_op
        for Ntau in ntaus:
            op = Operator(n, n, h, w["material"], Nt, Ntau, dt, w["p"], sink, q_time=qt, solve=solve)
            op.assemble(rho)
            buf = PassBuffers(op)
            for k in range(1, args.sweep_kmax + 1):
                if k > Ntau:
                    break
                t, (Th, g) = timed(lambda: parareal_pass(op, buf, k))
                rows.append(dict(design=dname, Ntau=Ntau, k=k, ms=t, sequential_ms=t_seq, speedup=t_seq / t,
                                 e_Theta=abs(float(Th.item()) - Th_s) / abs(Th_s),
                                 e_grad=float(torch.linalg.norm(g - g_s) / torch.linalg.norm(g_s))))
            del buf, op
    print(json.dumps({"metric": "k-iteration Parareal vs sequential FP64 GPU time stepping (paper test case)",
                      "config": {"workload": "paper100: 100x100, Nt=480, Table 1, q(t) of Eq. 5.1, bottom sink, p=20",
                                 "precision": "fp64", "rtol": 1e-12, "initial_guess": args.initial_guess,
                                 "coarse_propagator": "2h mesh (Sec. 7.3 future work)" if args.coarse_mesh else "h mesh"},
                      "paper_context": "MATLAB, CPU threads: Parareal speedup up to 5x at 16 threads with one iteration",
                      "rows": rows}), flush=True)


# ---------------------------------------------------------------------------- CPU oracle arms

ORACLE_SNIPPET = r"""
import json, os, sys, time
sys.path.insert(0, {root!r})
import numpy as np
import workloads as W
from oracle import Material, Operator, Problem
from oracle.parareal import F_pri, F_adj
w = W.workload('oneshot128')
n = w['n']; h = w['h']
prob = Problem(nx=n, ny=n, h=h, material=Material(**w['material']), Nt=w['Nt'], dt=w['dt'], Ntau=w['Ntau'],
               p=w['p'], dirichlet=W.dirichlet_left_centre(n, n, h))
rho = W.rho_warm_perturb(W.rho_uniform(n, n, 0, 0.2, 0.8), seed=1000, amp=0.01)
budget = {budget}
t0 = time.perf_counter()
op = Operator(prob, rho)
op._factor(prob.dt)
T = np.zeros(prob.Nn); theta = 0.0
steps = 0
s = 0
hist = np.zeros((prob.M + 1, prob.Nn))
while time.perf_counter() - t0 < budget and s < prob.Ntau:
    Tn, theta, inter = F_pri(op, s, T, theta)           # fine primal slice
    hist[0] = T; hist[1:] = inter
    full = np.zeros((prob.Nt + 1, prob.Nn)); full[prob.M * s: prob.M * (s + 1) + 1] = hist
    F_adj(op, s, np.zeros(prob.Nn), np.zeros(prob.Ne), full, max(theta, 1e-3))   # fine adjoint slice
    steps += 2 * prob.M
    T = Tn; s += 1
dt_s = time.perf_counter() - t0
nfree = int(op.free.sum())
print(json.dumps({{'value': nfree * steps / dt_s, 'seconds': dt_s, 'slices': s, 'fine_steps': steps}}))
"""


def cpu_baseline(budget_s: float) -> dict:
    """The oracle (as it stands) on one host core: fine primal + adjoint slices of the same
    workload until the time budget is spent; DOF*steps/s of that sample."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    code = ORACLE_SNIPPET.format(root=ROOT, budget=budget_s)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=budget_s * 10 + 120)
    if r.returncode != 0:
        return {"value": None, "unit": UNIT, "cores": 1, "kind": "oracle", "error": r.stderr[-300:]}
    d = json.loads(r.stdout.strip().splitlines()[-1])
    return {"value": d["value"], "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{d['slices']} fine primal + adjoint slices (M=32 steps each, {d['fine_steps']} fine solves) "
                      f"of the 128x128 workload, banded Cholesky, {d['seconds']:.1f} s, BLAS threads = 1"}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    budget = max(2.0, min(20.0, 150.0 / max(1, args.steps + args.warmup)))
    for _ in range(args.warmup):
        cpu_baseline(budget)
    vals = []
    t0 = time.perf_counter()
    for _ in range(args.steps):
        vals.append(cpu_baseline(budget))
    wall = time.perf_counter() - t0
    v = float(np.mean([x["value"] for x in vals if x["value"]])) if vals else None
    ms = wall / max(1, args.steps) * 1e3
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"{WORKLOAD}: 128x128 grid, Nt=1024, Ntau=32; bounded sample per step "
                                   f"({budget:.0f} s of fine primal+adjoint slices)"},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": vals[0]["sample"] if vals else None},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--precision", default="fp32_refine", choices=["fp32_refine", "fp32_refine_all", "fp64"],
                    help="fp32_refine: fine-step CG in FP32 with FP64 refinement, coarse-step solves FP64; "
                         "fp32_refine_all: every CG in FP32 with FP64 refinement")
    ap.add_argument("--rtol", type=float, default=1e-10)
    ap.add_argument("--twolevel", default="threelevel", choices=["none", "additive", "vcycle", "threelevel"],
                    help="preconditioner of the coarse-step solves: Jacobi, additive two-level, the "
                         "two-grid V(1,1) cycle, or the three-level cycle (2h Galerkin level and its aggregates)")
    ap.add_argument("--smooth", type=int, default=0,
                    help="V-cycle smoothing steps (1: one global Jacobi step; k >= 2: k slab-local steps; "
                         "0: the library default)")
    ap.add_argument("--local", type=int, default=0,
                    help="FP32 CG without two-level: 1 Jacobi, 2 two slab-local Jacobi steps, 0 the library default")
    ap.add_argument("--initial-guess", type=int, default=0,
                    help="CG starts of the time steps (ptg_solve.initial_guess): 1 plain, 2-4 extrapolated "
                         "through that many states, 0 the library default")
    ap.add_argument("--coarse-mesh", action="store_true",
                    help="--sweep / --loop: coarse propagators on the 2h mesh (Sec. 7.3 future work)")
    ap.add_argument("--sweep-ntau", default="5,10,16,20,30,32,48,60,80,96,120,160,240",
                    help="--sweep: slice counts (divisors of 480)")
    ap.add_argument("--sweep-kmax", type=int, default=8, help="--sweep: largest iteration count")
    ap.add_argument("--no-twolevel", dest="twolevel", action="store_const", const="none",
                    help="same as --twolevel none")
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    ap.add_argument("--no-extras", dest="extras", action="store_false",
                    help="time the passes only: no end-to-end run, comparator, accuracy checks or G = 0 probe "
                         "(for profiling the launch sequence of the timed steps)")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--coarse-stream", type=int, default=0, choices=[0, 1, 2],
                    help="coarse-step solves streamed with the multigrid V-cycle: 2 always, 1 never, "
                         "0 the library's choice (large grids)")
    ap.add_argument("--fine-stream", type=int, default=0, choices=[0, 1, 2],
                    help="fine propagators with their CG vectors in global memory, every slice at once "
                         "(ptg_solve.fine_stream): 2 always, 0/1 on chip")
    ap.add_argument("--no-overlap", dest="overlap", action="store_false",
                    help="run the adjoint coarse propagators after the forward correction sweep instead of as "
                         "two Theta-free parts beside it on a second stream")
    ap.add_argument("--no-c3", dest="c3", action="store_false",
                    help="leave out the 256x256 pass (Nt=2048, 64 slices) with its per-kernel roofline")
    ap.add_argument("--c3-steps", type=int, default=2, help="timed passes of the 256x256 line")
    ap.add_argument("--no-c4", dest="c4", action="store_false",
                    help="leave out the 48-design batching summary")
    ap.add_argument("--no-c5", dest="c5", action="store_false",
                    help="leave out the 512x512 design loop summary (3 design iterations)")
    ap.add_argument("--c3-workload", default="diff256", choices=["diff256", "loop512"],
                    help="--c3-only: the grid of the per-kernel line (256x256 or 512x512)")
    ap.add_argument("--c3-only", action="store_true",
                    help="only the 256x256 line (its JSON object), e.g. to capture its kernels under a profiler")
    ap.add_argument("--loop", type=int, default=0, metavar="ITERATIONS",
                    help="instead of the pass benchmark: the full design loop (512x512, Nt=4096, 128 slices, "
                         "host MMA) for this many design iterations")
    ap.add_argument("--loop-n", type=int, default=512, help="grid side of --loop")
    ap.add_argument("--sweep", action="store_true",
                    help="instead of the pass benchmark: k-iteration Parareal error / speedup sweep of the paper's "
                         "test case (100x100, Nt=480, Table 1, Eq. 5.1 load, bottom sink, p=20)")
    ap.add_argument("--batch48", action="store_true",
                    help="instead of the pass benchmark: the 48-design batching workload (persistent launches, "
                         "CUDA graph) against the same passes design by design")
    ap.add_argument("--autotune", action="store_true", help="--batch48: autotune every phase's plan first")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.batch48:
        run_batch48(args)
    elif args.loop:
        run_loop(args)
    elif args.sweep:
        run_sweep(args)
    elif args.c3_only:
        run_c3_only(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
