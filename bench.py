#!/usr/bin/env python
"""Benchmark: solves/s of recycled GMRES(m) over a convection-diffusion time-step sequence.

One bench step = one time step of Algorithm 1 on the device: new operator values
and right-hand side (assembled on the device from the previous solution, outside
the timed segment), then, timed with CUDA events on the solver's stream,
rgm_set_operator_values + rgm_solve + rgm_update_recycle_svd.  L2 is flushed
(256 MiB write) before every timed segment.  Default workload: Q4 elements on a
256 x 256 grid (1,050,625 dofs, 37.5 M nonzeros), eps 0.002, dt 0.002,
GMRES(40), k = 12 recycle vectors from a window of 24, true residual 1e-8; the
headline is deflated GMRES-IR (binary32 Arnoldi and projections inside a
binary64 refinement loop), with plain GMRES-IR and binary64 deflated, plain and
augmented GMRES measured on the same sequence.

Multi-GPU (torchrun): independent sequences per rank (replicas, no collective
on the data path); value = all ranks' solves / slowest rank's time.
--impl reference times the FP64 CPU oracle on the same workload instead.
"""
from __future__ import annotations

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

METRIC = "solves/s & HBM GB/s at ‖r‖/‖b‖≤1e-8: recycled vs plain GMRES(m); p99 latency"
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12      # 152 SMs x 2 FP64 FMA/clk x 2 flop x 2.07 GHz


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="q4_256x256_eps0.002_dt0.002",
                    help="a single-sequence workload, batch64 (64 uneven sequences solved together), "
                         "serve (a Poisson stream of sequences, continuous batching) or table2 "
                         "(extrapolated vs projection initial guesses on the paper's nu = 0.1 benchmark)")
    ap.add_argument("--mode", default="deflated", choices=["plain", "deflated", "augmented", "guess"])
    ap.add_argument("--grid", type=int, default=None,
                    help="override the workload's N (N x N quads), e.g. a smaller case of the same "
                         "kernels for a profiler capture")
    ap.add_argument("--k", type=int, default=None, help="override the workload's recycle dimension")
    ap.add_argument("--window", type=int, default=None, help="override the workload's snapshot window")
    ap.add_argument("--svd-interval", type=int, default=None, help="override the workload's SVD interval")
    ap.add_argument("--precond", default=None, choices=["none", "jacobi"],
                    help="override the workload's preconditioner")
    ap.add_argument("--precision", default="fp32_ir", choices=["fp64", "fp32_ir"])
    ap.add_argument("--cpu-steps", type=int, default=0, help="oracle steps for cpu_baseline (0: auto)")
    ap.add_argument("--quick", action="store_true", help="skip e2e, cpu baseline and side modes")
    ap.add_argument("--serve-count", type=int, default=512, help="serve: number of sequences")
    ap.add_argument("--serve-rate", type=float, default=0.0,
                    help="serve: mean arrivals per second (0: the rate that loads 80 %% of HBM)")
    ap.add_argument("--launch-policy", default="auto", choices=["auto", "per_pass"],
                    help="Arnoldi steps of a cycle in one cooperative launch (auto) or one launch per pass")
    ap.add_argument("--batch-policy", default="streams", choices=["coop", "streams"],
                    help="batch64 / serve: all systems' cycles in batched cooperative launches (coop) "
                         "or per-pass launches on the systems' streams")
    return ap.parse_args()


def dist_info():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def replica_sequence(rank):
    """Replicas (no data-path collective): rank r solves sequence r of the
    workload, an independent problem with its own seeded draws."""
    return rank


def aggregate_replicas(my_sec, steps, ws, reduce_max):
    """Whole-job throughput of ws replicas that each ran `steps` timed solves:
    the job lasts as long as the slowest rank (max over ranks through
    reduce_max), and all ranks' solves count.  Returns (value, job seconds)."""
    tot = reduce_max(my_sec) if ws > 1 else my_sec
    return steps * ws / tot, tot


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def src_digest():
    """Digest of the sources the Arnoldi-step kernels are built and launched
    from (the fused passes, their dispatch and the solver's launch geometry);
    the SVD, FE and allocation-free kernels are not part of it."""
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_1807_09467_gb300", "csrc")
    for f in sorted(os.listdir(d)):
        if f.startswith(("vec_", "common", "solver")):
            h.update(open(os.path.join(d, f), "rb").read())
    return h.hexdigest()[:16]


def traffic_record(workload, precision, kernel):
    """DRAM bytes per launch of `kernel` on this workload from the committed
    ncu summary, if it was taken on the current kernel sources; else None."""
    try:
        rec = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
    except Exception:
        return None
    ent = rec.get(f"{workload}/{precision}/{kernel}")
    if not ent or ent.get("src_sha") != src_digest():
        return None
    return ent.get("dram_bytes_per_launch")


class ClockSampler:
    """nvidia-smi samples during the timed region (SM clock, throttle reasons)."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


def iters_stats(its):
    its = [int(i) for i in its]
    return {"mean": round(statistics.mean(its), 2),
            "sd": round(statistics.pstdev(its), 2) if len(its) > 1 else 0.0}


# ------------------------------------------------------------------ workloads
def workload_fe(rg, w, beta, stream=None):
    """The workload's FE handle (Sec. 6.1's cellular velocity when it asks)."""
    fe = rg.FE(w.p, w.N, w.eps, w.dt, beta, stream=stream)
    if w.velocity == "cellular":
        fe.set_velocity("cellular")
    return fe


def workload_u0(np, fe, w, a8):
    return np.zeros(fe.n) if w.u0 == "zero" else fe.initial_field(a8)


def workload_of(synth, args):
    """The named workload with the command line's overrides applied."""
    import dataclasses
    w = synth.WORKLOADS[args.workload]
    over = {}
    if args.k is not None:
        over["k"] = args.k
    if args.window is not None:
        over["window"] = args.window
    if args.svd_interval is not None:
        over["ell"] = args.svd_interval
    if args.precond is not None:
        over["precond"] = args.precond
    if args.grid is not None:
        over["N"] = args.grid
        over["name"] = w.name.replace(f"{w.N}x{w.N}", f"{args.grid}x{args.grid}")
    return dataclasses.replace(w, **over) if over else w


def workload_seq(synth, w, index, steps):
    """(a8, beta, forcing rows or None) of one sequence."""
    a8, beta = synth.sequence_draws(w, index)
    forcing = synth.forcing_draws(w, steps, index) if w.forcing_modes else None
    return a8, beta, forcing


# ------------------------------------------------------------------ our arm
def run_sequence(rg, torch, w, seq, mode, precision, warmup, steps, profile=False, keep=None,
                 flush=None, stream=None, guess=0, keep_x=0):
    """Runs warmup + steps time steps on the device; returns timing and stats
    (and the solutions of the first keep_x steps, on the host)."""
    import numpy as np
    a8, beta, forcing = seq
    dev = torch.device("cuda")
    fe = workload_fe(rg, w, beta, stream=stream)
    rp, col = fe.pattern()
    rtol = w.rtol if precision == "fp64" else 1e-8
    solver = rg.Solver(fe.n, m=w.m, k=w.k, window=w.window, svd_interval=w.ell, mode=mode,
                       precision=precision, rtol=rtol, stream=stream, launch_policy=LAUNCH_POLICY[0],
                       precond=w.precond, guess=guess)
    u0 = workload_u0(np, fe, w, a8)
    u = torch.tensor(u0, dtype=torch.float64, device=dev)
    solver.set_operator_csr(rp, col, torch.zeros(len(col), dtype=torch.float64).numpy())
    x = torch.empty_like(u)
    cs = torch.cuda.current_stream()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(warmup + steps)]
    eva = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(warmup + steps)]
    its, res, kus, refs, xs = [], [], [], [], []
    prof = None
    for i in range(warmup + steps):
        if i == warmup and profile:
            solver.profile(True)
        if forcing is not None:
            fe.set_forcing(forcing[i], w.forcing_C)
        eva[i][0].record(cs)
        val, b = fe.assemble(u)                         # workload step, not timed
        eva[i][1].record(cs)
        if keep is not None:
            keep.append((val.cpu(), b.cpu()))
        zg = solver.recycle_dim() > 0 and mode != "plain"     # x_in = 0: x0 = U E^-1 U^T b
        if not zg:
            x.copy_(u)
        if flush is not None:
            flush.zero_()
        ev[i][0].record(cs)
        solver.set_operator_values(val)
        _, st = solver.solve(b, x, zero_guess=zg)
        solver.update_recycle_svd(x, want_k=False)
        ev[i][1].record(cs)
        u.copy_(x)
        its.append(st["iters"])
        res.append(st["true_relres"])
        kus.append(st["k_used"])
        refs.append(st["refinements"])
        if i < keep_x:
            xs.append(x.cpu().numpy())
    torch.cuda.synchronize()
    if profile:
        prof = solver.profile_read()
        solver.profile(False)
    seg = [ev[i][0].elapsed_time(ev[i][1]) for i in range(warmup + steps)]
    asm = [eva[i][0].elapsed_time(eva[i][1]) for i in range(warmup + steps)]
    solver.close()
    fe.close()
    return dict(seg_ms=seg[warmup:], asm_ms=asm[warmup:], iters=its, relres=res, k_used=kus,
                refinements=refs, x_first=xs, prof=prof, n=fe.n, nnz=len(col),
                u_final=u.cpu().numpy())


def run_e2e(rg, np, w, seq, mode, precision, warmup, steps, inputs, torch):
    """Same sequence through the public API with host (pinned) buffers."""
    a8, beta, _ = seq
    n = len(inputs[0][1])
    fe = workload_fe(rg, w, beta)
    rp, col = fe.pattern()
    u = workload_u0(np, fe, w, a8)
    fe.close()
    rtol = w.rtol if precision == "fp64" else 1e-8
    s = rg.Solver(n, m=w.m, k=w.k, window=w.window, svd_interval=w.ell, mode=mode,
                  launch_policy=LAUNCH_POLICY[0],
                  precision=precision, rtol=rtol, precond=w.precond)
    s.set_operator_csr(rp, col, np.zeros(len(col)))
    pin_val = torch.empty(len(col), dtype=torch.float64).pin_memory()
    pin_b = torch.empty(n, dtype=torch.float64).pin_memory()
    pin_x = torch.empty(n, dtype=torch.float64).pin_memory()
    times, h2d = [], []
    for i in range(warmup + steps):
        val, b = inputs[i]
        pin_val.copy_(val)
        pin_b.copy_(b)
        zg = s.recycle_dim() > 0 and mode != "plain"
        if not zg:
            pin_x.copy_(torch.from_numpy(u))
        t0 = time.perf_counter()
        s.set_operator_values(pin_val.numpy())
        xx, st = s.solve(pin_b.numpy(), pin_x.numpy(), zero_guess=zg)
        s.update_recycle_svd(xx, want_k=False)
        t1 = time.perf_counter()
        u = xx
        times.append(t1 - t0)
        # values, b, x_in (unless zero), and x again for the window update
        h2d.append(8 * len(col) + 8 * n * (2 + (0 if zg else 1)))
    s.close()
    return dict(sec=times[warmup:], h2d=int(statistics.mean(h2d[warmup:])), d2h=8 * n)


LAUNCH_POLICY = ["auto"]


def fp64_peak_tflops(torch):
    """Measured binary64 throughput of this GPU: cuBLAS DGEMM (torch.matmul on
    float64, 4096^3, 2 n^3 flops), best of 5 after 2 warm-ups, CUDA events."""
    n = 4096
    a = torch.randn(n, n, dtype=torch.float64, device="cuda")
    b = torch.randn(n, n, dtype=torch.float64, device="cuda")
    best = float("inf")
    for i in range(7):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        torch.matmul(a, b)
        e1.record()
        torch.cuda.synchronize()
        if i >= 2:
            best = min(best, e0.elapsed_time(e1) / 1e3)
    del a, b
    return 2.0 * n ** 3 / best / 1e12


def fp32_peak_tflops(torch):
    """Binary32 CUDA-core peak derived from the unit counts: SMs x 128 FP32
    lanes x 2 flops per FMA x the maximum SM clock (MEASURED_PEAKS.json
    sm_max_mhz, else 2070 MHz)."""
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    mhz = measured_peaks().get("sm_max_mhz", 2070.0)
    return sms * 128 * 2 * mhz * 1e6 / 1e12


ARNOLDI_PASSES = ("arnoldi_spmv_dots", "arnoldi_cgs1_axpy_dots", "arnoldi_cgs2_axpy_norm")


def cycle_roofline(prof, w, precision, hbm_peak, fp64_peak, fp32_peak=None):
    """Roofline of the Arnoldi step, the dominant kernel: the cooperative cycle
    launch, or the three fused-pass launches of each step.  Bytes are the
    algorithmic bytes of the steps, B_j = (e + 4) nnz + e n (j + 2 k + 4)
    summed over the steps (step_bytes, booked by the library), time the
    kernels' CUDA-event durations on the solver's stream; flops those of the
    passes (2 per nonzero, 2 per row per dot or AXPY column)."""
    kinds = {k: v for k, v in prof.items() if v["launches"] > 0}
    cyc = kinds.get("arnoldi_cycle")
    if cyc:
        parts = {"arnoldi_cycle": cyc}
        name = "arnoldi_cycle (cooperative launch of a cycle's Arnoldi steps)"
    else:
        parts = {k: kinds[k] for k in ARNOLDI_PASSES if k in kinds}
        name = "arnoldi_step (" + " + ".join(parts) + ", one launch each per step)"
    ms = sum(v["ms"] for v in parts.values())
    steps = sum(v["units"] for v in parts.values())
    sbytes = sum(v["step_bytes"] for v in parts.values())
    flops = sum(v["flops"] for v in parts.values())
    pbytes = sum(v["bytes"] for v in parts.values())
    t = ms * 1e-3 / steps
    gbs = sbytes / steps / t / 1e9
    tfl = flops / steps / t / 1e12
    hbm = {"bound": "hbm", "achieved": round(gbs, 1), "peak": hbm_peak, "unit": "GB/s",
           "frac": round(gbs / hbm_peak, 4),
           "peak_source": "of measured (MEASURED_PEAKS.json hbm_gbs, copy)"}
    if precision == "fp32_ir" and fp32_peak:
        # the passes' arithmetic is binary32 (binary64 only in the dot accumulators)
        alu = {"bound": "alu", "achieved": round(tfl, 4), "peak": round(fp32_peak, 2), "unit": "TFLOP/s",
               "frac": round(tfl / fp32_peak, 4),
               "peak_source": "derived: SMs x 128 FP32 lanes x 2 x maximum SM clock"}
    else:
        alu = {"bound": "alu", "achieved": round(tfl, 4), "peak": round(fp64_peak, 4), "unit": "TFLOP/s",
               "frac": round(tfl / fp64_peak, 4),
               "peak_source": "of measured (cuBLAS DGEMM in this run, the binary64 pipe)"}
    head = hbm if precision == "fp32_ir" else alu
    other = alu if precision == "fp32_ir" else hbm
    out = dict(head)
    out.update({"kernel": name, "unit_of_work": "one Arnoldi step", "steps": int(steps),
                "ms_per_step": round(t * 1e3, 5),
                "algorithmic_bytes_per_step": sbytes / steps,
                "algorithmic_flops_per_step": flops / steps,
                "pass_bytes_per_step": pbytes / steps,
                "pass_gbs": round(pbytes / steps / t / 1e9, 1),
                "per_pass": {k: {"launches": v["launches"], "us_per_launch": round(1e3 * v["ms"] / v["launches"], 2),
                                 "gbs": round(v["bytes"] / (v["ms"] * 1e-3) / 1e9, 1)}
                             for k, v in parts.items()},
                "traffic": traffic_record(w.name, precision, "arnoldi_step"),
                "second_bound": other})
    return out, kinds


def ours(args):
    LAUNCH_POLICY[0] = args.launch_policy
    import numpy as np
    import torch

    import __graft_entry__ as g
    import paper_1807_09467_gb300 as rg
    import synth

    ws, rank, local = dist_info()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        if rank == 0:
            g.build()
        dist.barrier()
    else:
        g.build()
    w = workload_of(synth, args)
    seq = workload_seq(synth, w, replica_sequence(rank), max(w.steps, args.warmup + args.steps))
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")   # 256 MiB
    S = cpu_sample_steps(args, w)

    keep = [] if (rank == 0 and not args.quick) else None
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clk = ClockSampler(local)
    clk.start()
    t_wall0 = time.perf_counter()
    main = run_sequence(rg, torch, w, seq, args.mode, args.precision, args.warmup, args.steps,
                        profile=False, keep=keep, flush=flush, keep_x=0 if args.quick else S)
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall0
    clocks = clk.stop()
    # second pass over the same sequence with per-launch CUDA events on the
    # solver's stream (events between launches serialise the overlap of
    # consecutive passes, so this pass is not the headline timing)
    profd = run_sequence(rg, torch, w, seq, args.mode, args.precision, args.warmup, args.steps,
                         profile=True, flush=flush)
    my_sec = sum(main["seg_ms"]) / 1e3

    def reduce_max(x):
        t = torch.tensor([x], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    K = args.steps
    value, tot_sec = aggregate_replicas(my_sec, K, ws, reduce_max)
    if ws > 1:
        dist.barrier()
    if rank != 0:
        if ws > 1:
            dist.destroy_process_group()
        return
    prof, launches = profd["prof"]
    n, nnz = main["n"], main["nnz"]
    peaks = measured_peaks()
    hbm_peak = peaks.get("hbm_gbs", 6690.5)
    fp64_peak = fp64_peak_tflops(torch)
    fp32_peak = fp32_peak_tflops(torch)
    roof, kinds = cycle_roofline(prof, w, args.precision, hbm_peak, fp64_peak, fp32_peak)
    tot_ms = sum(v["ms"] for v in kinds.values())
    kernel_share = {k: {"ms": round(v["ms"], 3), "share": round(v["ms"] / tot_ms, 4),
                        "launches": v["launches"]} for k, v in kinds.items()}
    seg = main["seg_ms"]
    rtol = w.rtol if args.precision == "fp64" else 1e-8
    out = {
        "metric": METRIC, "value": round(value, 3), "unit": "solves/s", "n_gpus": ws, "steps": K,
        "warmup": args.warmup, "ms_per_step": round(tot_sec * 1e3 / K, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f32+f64",
        "data": "synthetic",
        "config": {"workload": w.name, "n": n, "nnz": nnz, "p": w.p, "N": w.N, "m": w.m, "k": w.k,
                   "window": w.window, "svd_interval": w.ell, "mode": args.mode,
                   "velocity": w.velocity, "forcing_modes": w.forcing_modes, "u0": w.u0,
                   "precond": w.precond,
                   "precision": args.precision, "launch_policy": args.launch_policy,
                   "rtol": rtol, "true_residual": "||b - A x|| / ||b|| in binary64",
                   "l2": "flushed (256 MiB write) before every timed step",
                   "parallelism": "replicas" if ws > 1 else "single"},
        "latency_ms": {"p50": round(float(np.percentile(seg, 50)), 4),
                       "p99": round(float(np.percentile(seg, 99)), 4)},
        "iterations": iters_stats(main["iters"][args.warmup:]),
        "refinements": iters_stats(main["refinements"][args.warmup:]),
        "max_true_relres": max(main["relres"][args.warmup:]),
        "assembly_ms_per_step": round(statistics.mean(main["asm_ms"]), 4),
        "roofline": roof, "kernels": kernel_share, "gpu_launches": int(launches),
        "profiled_pass_ms_per_step": round(statistics.mean(profd["seg_ms"]), 4),
        "fp64_peak_tflops_measured": round(fp64_peak, 4),
        "clocks": clocks, "wall_s": round(t_wall, 3),
    }
    if not args.quick:
        # recycled vs plain and mixed vs binary64 on the same sequence
        side = {}
        for prec, md in (("fp32_ir", "deflated"), ("fp32_ir", "plain"), ("fp64", "deflated"),
                         ("fp64", "plain"), ("fp64", "augmented")):
            if (prec, md) == (args.precision, args.mode):
                r = main
            else:
                r = run_sequence(rg, torch, w, seq, md, prec, args.warmup, K, flush=flush)
            side[f"{prec}/{md}"] = {"solves_per_s": round(K / (sum(r["seg_ms"]) / 1e3), 3),
                                    "ms_per_step": round(statistics.mean(r["seg_ms"]), 4),
                                    "iterations": iters_stats(r["iters"][args.warmup:]),
                                    "max_true_relres": max(r["relres"][args.warmup:])}
        out["modes"] = side
        # the binary64 deflated cycle kernel on the roofline too (binary64 pipe)
        other_prec = "fp64" if args.precision == "fp32_ir" else "fp32_ir"
        r64 = run_sequence(rg, torch, w, seq, args.mode, other_prec, args.warmup, min(K, 10),
                           profile=True, flush=flush)
        out["roofline_" + other_prec], _ = cycle_roofline(r64["prof"][0], w, other_prec, hbm_peak,
                                                          fp64_peak, fp32_peak)
        # end to end through the public API with host buffers
        e = run_e2e(rg, np, w, seq, args.mode, args.precision, args.warmup, K, keep, torch)
        out["e2e"] = {"value": round(K / sum(e["sec"]), 3), "unit": "solves/s",
                      "h2d_bytes_per_step": e["h2d"], "d2h_bytes_per_step": e["d2h"]}
        # CPU baseline: the oracle on a bounded sample of the same sequence
        out["cpu_baseline"], out["parity"] = cpu_baseline(args, w, seq, main, np, S)
    print(json.dumps(out))
    if ws > 1:
        dist.destroy_process_group()


def run_batch(args):
    """Batched form: 64 independent sequences of uneven size (synth.batch_sequences)
    advanced one time step at a time; per step every sequence's operator is
    assembled (outside the timed region), then timed on the device: new
    values, one rgm_batch_solve over all 64 handles (each on its own stream),
    and the window updates.  Both batch policies are measured (the systems'
    cycles in batched cooperative launches, or per-pass launches on their
    streams); the same steps solved one handle after another give the
    sequential figure."""
    import numpy as np
    import torch

    import __graft_entry__ as g
    import paper_1807_09467_gb300 as rg
    import synth
    g.build()
    from paper_1807_09467_gb300 import tune
    seqs = synth.batch_sequences(64)
    prec = args.precision
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")

    def setup(cap=None):
        st = []
        for w, a8, beta in seqs:
            stream = torch.cuda.Stream()
            fe = rg.FE(w.p, w.N, w.eps, w.dt, beta, stream=stream.cuda_stream)
            rp, col = fe.pattern()
            sol = rg.Solver(fe.n, m=w.m, k=w.k, window=w.window, mode=args.mode, precision=prec,
                            rtol=w.rtol, stream=stream.cuda_stream,
                            tiles_per_block=tune.tiles_per_block(fe.n, cap))
            sol.set_operator_csr(rp, col, np.zeros(len(col)))
            u = torch.tensor(fe.initial_field(a8), dtype=torch.float64, device="cuda")
            st.append(dict(fe=fe, sol=sol, u=u, stream=stream, val=None, b=None))
        return st

    def step(state, batched, coop):
        for e in state:                                   # assembly: outside the timed region
            e["val"], e["b"] = e["fe"].assemble(e["u"])
            # initial guess: zero with a recycle space (x0 = U E^-1 U^T b), else x_{i-1}
            e["x"] = torch.zeros_like(e["u"]) if e["sol"].recycle_dim() else e["u"].clone()
        torch.cuda.synchronize()
        flush.zero_()
        torch.cuda.synchronize()
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record()
        for e in state:
            e["sol"].set_operator_values(e["val"])
        if batched:
            stats = rg.batch_solve([e["sol"] for e in state], [e["b"] for e in state],
                                   [e["x"] for e in state], coop=coop)
        else:
            stats = [e["sol"].solve(e["b"], e["x"])[1] for e in state]
        for e in state:
            e["sol"].update_recycle_svd(e["x"], want_k=False)
        cur = torch.cuda.current_stream()
        for e in state:
            cur.wait_stream(e["stream"])
        t1.record()
        torch.cuda.synchronize()
        for e in state:
            e["u"].copy_(e["x"])
        return t0.elapsed_time(t1), stats

    def run_arm(batched, coop, cap, warmup, steps):
        state = setup(cap)
        ms, its = [], []
        for i in range(warmup + steps):
            t, stats = step(state, batched, coop)
            assert all(st["status"] == 0 and st["true_relres"] <= 1e-8 for st in stats), stats
            if i >= warmup:
                ms.append(t)
                its.extend(st["iters"] for st in stats)
        for e in state:
            e["sol"].close()
            e["fe"].close()
        del state
        torch.cuda.synchronize()
        return ms, its

    # autotuner: the cap on the blocks of any one system (more 256-row tiles a
    # block), trial = the mean batch step of the chosen policy over steps
    # 4..5 of the sequences; the default (no cap) is listed first
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    caps = [None, 2 * nsm, nsm, nsm // 2]
    policy_coop = args.batch_policy == "coop"
    best, trials = tune.tune(lambda c: statistics.mean(run_arm(True, policy_coop, c, 3, 2)[0]), caps)
    out = {}
    for arm, batched, coop in (("coop", True, True), ("streams", True, False), ("sequential", False, False)):
        out[arm] = run_arm(batched, coop, best if batched and coop == policy_coop else None,
                           args.warmup, args.steps)
    untuned = run_arm(True, policy_coop, None, args.warmup, args.steps) if best is not None else None
    other = "streams" if args.batch_policy == "coop" else "coop"
    ms, its = out[args.batch_policy]
    mso, _ = out[other]
    mss, _ = out["sequential"]
    K = args.steps
    value = 64 * K / (sum(ms) / 1e3)
    res = {"metric": METRIC, "value": round(value, 3), "unit": "solves/s", "n_gpus": 1, "steps": K,
           "warmup": args.warmup, "ms_per_step": round(sum(ms) / K, 4), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64" if prec == "fp64" else "f32+f64",
           "data": "synthetic",
           "config": {"workload": "batch64: 64 independent sequences, Q1-Q4 on 32^2..192^2 quads, "
                                  "eps 10^U(-3,-1), one time step of every sequence per step",
                      "total_dofs": int(sum(w.n for w, _, _ in seqs)), "mode": args.mode,
                      "precision": prec, "m": 30, "k": 8, "window": 16, "rtol": 1e-8,
                      "l2": "flushed (256 MiB write) before every timed step",
                      "parallelism": "rgm_batch_solve, one stream per sequence",
                      "batch_policy": args.batch_policy},
           "iterations": iters_stats(its),
           other: {"solves_per_s": round(64 * K / (sum(mso) / 1e3), 3), "ms_per_step": round(sum(mso) / K, 4)},
           "sequential": {"solves_per_s": round(64 * K / (sum(mss) / 1e3), 3),
                          "ms_per_step": round(sum(mss) / K, 4)},
           "speedup_vs_sequential": round(sum(mss) / sum(ms), 3),
           "autotune": {"knob": "cap on the blocks of one system (tiles_per_block of each handle)",
                        "chosen_max_blocks": best,
                        "trial_ms_per_batch_step": {str(c): round(t, 3) for c, t in trials.items()},
                        "untuned_solves_per_s": (round(64 * K / (sum(untuned[0]) / 1e3), 3)
                                                 if untuned else round(value, 3))}}
    print(json.dumps(res))


def serve_rate(serve, reqs, hbm_gbs, load=0.8, iters=25):
    """Arrival rate (sequences per second) that loads `load` of the HBM
    bandwidth: each solve is predicted to move `iters` Arnoldi steps of
    binary32 GMRES-IR, (4 + 4) nnz + 4 n (m/2 + 2 k + 4) bytes a step; a
    sequence moves that times its steps."""
    def seq_bytes(r):
        n, nnz = serve.sizes(r.p, r.N)
        return r.steps * iters * (8.0 * nnz + 4.0 * n * (r.m / 2 + 2 * r.k + 4))
    mean = sum(seq_bytes(r) for r in reqs) / len(reqs)
    return load * hbm_gbs * 1e9 / mean


def run_serve(args):
    """Served form (config: 512 sequences, Q1-Q4 on 16^2..256^2 quads, eps
    log-uniform in [1e-3, 1e-1], 10-100 steps each, seeded Poisson arrivals):
    continuous batching (paper_1807_09467_gb300.serve), deflated GMRES-IR to a
    true residual of 1e-8, against plain binary64 GMRES(m) served by the same
    loop at the same arrivals.  The arrival rate loads the server at 80 %: the
    closed-loop capacity of the server (sequences per second with every request
    waiting at time 0) is measured on the first 64 requests and the Poisson rate
    set to 0.8 of it; the rate that would load 80 % of the HBM bandwidth by the
    bytes model (serve_rate) is reported beside it.  Solves/s and p50/p99
    per-solve latency (first solve of a sequence: from its arrival)."""
    import dataclasses

    import numpy as np
    import torch

    import __graft_entry__ as g
    import synth
    g.build()
    from paper_1807_09467_gb300 import serve
    hbm = measured_peaks().get("hbm_gbs", 6690.5)
    base = [serve.Request(**r) for r in synth.serve_stream(count=args.serve_count, rate_per_s=1.0,
                                                            n_hi=256)]
    hbm_rate = serve_rate(serve, base, hbm)
    # closed-loop capacity of the deflated GMRES-IR server on the first 64 requests
    cal = [dataclasses.replace(r, arrival_s=0.0) for r in base[:64]]
    # launch-shape autotuner: the closed-loop wall time of those requests for
    # each cap on the blocks of one sequence; the fastest cap serves both arms
    nsm = torch.cuda.get_device_properties(0).multi_processor_count

    def cal_wall(cap):
        _, t = serve.Server(max_slots=64, precision="fp32_ir", mode="deflated", max_blocks=cap).run(
            cal, realtime=False)
        return 1e3 * t["wall_s"]
    from paper_1807_09467_gb300 import tune
    cal_wall(None)                      # untimed: first-use costs out of the trials
    cap, cal_trials = tune.tune(cal_wall, [None, 2 * nsm, nsm])
    capacity = len(cal) / (cal_trials[cap] / 1e3)
    rate = args.serve_rate or 0.8 * capacity
    reqs = [dataclasses.replace(r, arrival_s=r.arrival_s / rate) for r in base]
    torch.cuda.synchronize()
    res, tot = serve.Server(max_slots=64, precision="fp32_ir", mode="deflated", max_blocks=cap).run(
        reqs, realtime=True)
    torch.cuda.synchronize()
    bres, btot = serve.Server(max_slots=64, precision="fp64", mode="plain", max_blocks=cap).run(
        reqs, realtime=True)
    its = [i for r in res for i in r.iters]
    bits = [i for r in bres for i in r.iters]
    first = [r.latencies_ms[0] for r in res if r.latencies_ms]
    later = [x for r in res for x in r.latencies_ms[1:]]
    pct = lambda v, q: round(float(np.percentile(v, q)), 3) if v else None
    out = {"metric": METRIC, "value": round(tot["solves_per_s"], 3), "unit": "solves/s", "n_gpus": 1,
           "steps": tot["solves"], "warmup": 0, "ms_per_step": round(1e3 * tot["wall_s"] / tot["solves"], 4),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
           "data": "synthetic",
           "config": {"workload": f"serve: {len(reqs)} sequences, Q1-Q4 on 16^2..256^2 quads, 10-100 steps, "
                                  f"Poisson arrivals at {rate:.2f} sequences/s (80 % of the server's measured "
                                  "capacity), deflated GMRES-IR to 1e-8, continuous batching (64 slots, 80 % of "
                                  "free HBM)",
                      "requests": len(reqs), "solves": tot["solves"], "arrival_rate_per_s": rate,
                      "capacity_sequences_per_s": round(capacity, 3),
                      "hbm_rule_rate_per_s": round(hbm_rate, 3), "hbm_gbs_for_rate": hbm},
           "latency_ms": {"p50": round(tot["p50_ms"], 3), "p99": round(tot["p99_ms"], 3),
                          "first_solve_p50": pct(first, 50), "first_solve_p99": pct(first, 99),
                          "later_solves_p50": pct(later, 50), "later_solves_p99": pct(later, 99)},
           "iterations": iters_stats(its), "wall_s": round(tot["wall_s"], 3),
           "autotune": {"knob": "cap on the blocks of one sequence (tiles_per_block of each handle)",
                        "chosen_max_blocks": cap,
                        "trial_ms_64_requests_closed_loop": {str(c): round(t, 1) for c, t in cal_trials.items()}},
           "footprint_estimate_over_measured": tot["footprint_estimate_over_measured"],
           "plain_fp64_same_loop": {"solves_per_s": round(btot["solves_per_s"], 3),
                                    "p50_ms": round(btot["p50_ms"], 3), "p99_ms": round(btot["p99_ms"], 3),
                                    "wall_s": round(btot["wall_s"], 3), "iterations": iters_stats(bits)}}
    print(json.dumps(out))


def run_table2(args):
    """Table 2's comparison on the device (Sec. 6.1 benchmark, nu = 0.1, no
    SSOR): for s = 2, 3, 4 the extrapolated guess from s solutions (Eq.
    ext2-ext4, GMRES(30) on A) against the projection guess with s recycled
    modes (Sec. 4.2, RGM_GUESS, GMRES(30) on A); iterations over the timed
    steps, and deflation with the same s for reference."""
    import dataclasses
    import torch

    import __graft_entry__ as g
    import paper_1807_09467_gb300 as rg
    import synth
    g.build()
    w0 = synth.PAPER_Q1_64[0.1]
    W, K = args.warmup, args.steps
    seq = workload_seq(synth, w0, 0, max(w0.steps, W + K))
    rows = []
    for s_ in (2, 3, 4):
        row = {"s": s_}
        for name, mode, guess, k in (("ext", "plain", s_ - 1, 0), ("proj", "guess", 0, s_),
                                     ("def", "deflated", 0, s_)):
            w = dataclasses.replace(w0, k=k)
            r = run_sequence(rg, torch, w, seq, mode, "fp64", W, K, guess=guess)
            row[name] = {"iterations": iters_stats(r["iters"][W:]),
                         "solves_per_s": round(K / (sum(r["seg_ms"]) / 1e3), 3)}
        rows.append(row)
    out = {"metric": METRIC, "value": rows[-1]["proj"]["solves_per_s"], "unit": "solves/s", "n_gpus": 1,
           "steps": K, "warmup": W, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f64", "data": "synthetic",
           "config": {"workload": f"table2: {w0.name}, GMRES(30), window 16, steps {W + 1}..{W + K}"},
           "table2": rows}
    print(json.dumps(out))


def cpu_sample_steps(args, w):
    """Oracle time steps that make about 10-30 s of CPU work: high-order
    assembly costs (p+1)^6 per cell, a 1 M-dof step about 20 s."""
    return args.cpu_steps or min(w.steps, 2 if w.p > 4 else 30 if w.n < 200000 else 2)


def oracle_sequence(orc, w, seq_i, S, mode, precision, keep_all=False):
    a8, beta, forcing = seq_i
    import numpy as np
    u0 = np.zeros(w.n) if w.u0 == "zero" else orc.u0_field(w.p, w.N, a8)
    rtol = w.rtol if precision == "fp64" else 1e-8
    return orc.sequence(w.p, w.N, w.eps, w.dt, beta, S, u0, mode=mode, m=w.m, k=w.k,
                        window=w.window, ell=w.ell, rtol=rtol, keep_all=keep_all,
                        velocity=int(w.velocity == "cellular"), forcing=forcing,
                        forcing_C=w.forcing_C, precond=int(w.precond == "jacobi"),
                        precision=int(precision == "fp32_ir"), inner_rtol=1e-4, inner_cycles=2)


def cpu_baseline(args, w, seq, main, np, S):
    import oracle as orc
    orc.build()
    mode = {"plain": 0, "deflated": 1, "augmented": 2, "guess": 3}[args.mode]
    r = oracle_sequence(orc, w, seq, S, mode, args.precision, keep_all=True)
    secs = r["step_seconds"]
    kind = "GMRES-IR (binary32 inner storage, binary64 residual)" if args.precision == "fp32_ir" else "binary64"
    cb = {"value": round(S / float(secs.sum()), 4), "unit": "solves/s", "cores": 1, "kind": "oracle",
          "sample": f"first {S} time steps of the same sequence ({w.name}, {args.mode}, {kind}), "
                    f"FE assembly + solve + window SVD per step, single thread"}
    # the same oracle on every host core: independent sequences (their own
    # seeded draws), one per thread; the C oracle holds no global state and
    # its ctypes calls release the interpreter lock
    import os
    import synth
    from concurrent.futures import ThreadPoolExecutor
    ncores = os.cpu_count() or 1
    S1 = 1 if w.n >= 200000 else S

    def one(idx):
        ri = oracle_sequence(orc, w, workload_seq(synth, w, 1000 + idx, S1), S1, mode, args.precision)
        return int(ri["iters"].sum())

    t0 = time.perf_counter()
    with ThreadPoolExecutor(max_workers=ncores) as ex:
        list(ex.map(one, range(ncores)))
    wall = time.perf_counter() - t0
    cb["all_cores"] = {"value": round(ncores * S1 / wall, 4), "unit": "solves/s", "cores": ncores,
                       "kind": "oracle",
                       "sample": f"{ncores} independent sequences of {w.name} ({args.mode}, {kind}), "
                                 f"{S1} time steps each, one thread per sequence"}
    # parity on the steps both ran: iterations, refinements and x per step
    S2 = min(S, len(main["iters"]), len(main["x_first"]))
    gi = np.array(main["iters"][:S2])
    oi = np.array(r["iters"][:S2])
    xerr = [float(np.linalg.norm(main["x_first"][i] - r["x_all"][:, i]) / np.linalg.norm(r["x_all"][:, i]))
            for i in range(S2)]
    par = {"steps_compared": S2,
           "oracle_iterations": [int(v) for v in oi], "gpu_iterations": [int(v) for v in gi],
           "max_abs_iter_diff": int(np.max(np.abs(gi - oi))) if S2 else None,
           "max_rel_x_err": max(xerr) if xerr else None, "rel_x_err_per_step": xerr,
           "oracle_true_relres": [float(v) for v in r["relres"][:S2]],
           "gpu_true_relres": [float(v) for v in main["relres"][:S2]]}
    if args.precision == "fp32_ir":
        gr = np.array(main["refinements"][:S2])
        orf = np.array(r["refinements"][:S2])
        par.update({"oracle_refinements": [int(v) for v in orf], "gpu_refinements": [int(v) for v in gr],
                    "max_abs_refinement_diff": int(np.max(np.abs(gr - orf))) if S2 else None})
    return cb, par


# ------------------------------------------------------------------ reference arm
def reference(args):
    ws, rank, local = dist_info()
    if rank != 0:
        return
    import oracle as orc
    import synth
    orc.build()
    w = workload_of(synth, args)
    seq = workload_seq(synth, w, 0, max(w.steps, args.warmup + args.steps))
    # each bench step is one time step; the oracle is slow, so a step is a
    # bounded sample (the first warmup+steps steps of the sequence, capped)
    W, K = args.warmup, args.steps
    cap = 3 if w.p > 4 else 40 if w.n < 200000 else 3
    tot = min(W + K, cap)
    Wc = min(W, max(tot - 1, 0))
    Kc = tot - Wc
    mode = {"plain": 0, "deflated": 1, "augmented": 2, "guess": 3}[args.mode]
    r = oracle_sequence(orc, w, seq, tot, mode, args.precision)
    rtol = w.rtol if args.precision == "fp64" else 1e-8
    secs = r["step_seconds"][Wc:]
    value = Kc / float(secs.sum())
    kind = "GMRES-IR oracle (binary32 inner storage)" if args.precision == "fp32_ir" else "FP64 oracle"
    sample = (f"time steps {Wc + 1}..{tot} of the {w.name} sequence ({args.mode}), {kind}, "
              f"single thread")
    out = {"metric": METRIC, "value": round(value, 4), "unit": "solves/s", "n_gpus": args.gpus,
           "steps": Kc, "warmup": Wc, "ms_per_step": round(1e3 * float(secs.mean()), 3),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f64" if args.precision == "fp64" else "f32+f64",
           "data": "synthetic", "impl": "reference",
           "config": {"workload": w.name, "n": w.n, "m": w.m, "k": w.k, "window": w.window,
                      "mode": args.mode, "precision": args.precision, "rtol": rtol},
           "iterations": iters_stats(r["iters"][Wc:]),
           "cpu_baseline": {"value": round(value, 4), "unit": "solves/s", "cores": 1,
                            "kind": "oracle", "sample": sample},
           "e2e": {"value": round(value, 4), "unit": "solves/s", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


if __name__ == "__main__":
    a = parse()
    if a.impl == "reference":
        reference(a)
    elif a.workload == "batch64":
        run_batch(a)
    elif a.workload == "serve":
        run_serve(a)
    elif a.workload == "table2":
        run_table2(a)
    else:
        ours(a)
