#!/usr/bin/env python3
"""Benchmark of the directional splitting solver on one GB300.

Workload: the sheared-flow stationary problem on the unit square, 2048 x 2048
nodes, beta = (1, 0.5 + 0.3 sin 2 pi x), mu = 1e-3, sigma = 1, f = 8 seeded
Gaussians of width 0.02 (synthetic data), solved from u = 0 until the relative
update |u_{j+1} - u_j| / |u_{j+1}| <= 1e-8.

One step = one such solve.  value = line unknowns solved per second (both curve
families, every split step) over the timed steps; ms_per_step = time to 1e-8.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--prec fp64|fp32]
  python bench.py --transfer direct    # values between the curve families through
                                       # their crossings instead of the grid
  python bench.py --impl reference     # the FP64 CPU oracle on the same workload

With N > 1 (torchrun) every rank solves its own copy of the problem (the
path has no exchange step between independent problems): weak scaling, no
collective on the data path; the barrier and the max-over-ranks time only.
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

METRIC = "line-DOF/s (2D ADR directional splitting, time-to-1e-8 relative update)"
UNIT = "line-DOF/s"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM_GBS = 6800.0
# FP64 arithmetic peak of one GB300: 152 SMs x 2 FP64 FMA/clk (4 flop) x 2.07 GHz
FP64_PEAK_TFLOPS = 152 * 4 * 2.07e9 / 1e12

# Algorithmic traffic and FP64 work per unit of each sweep kernel in FP64 mode
# (unit = one curve unknown for the curve solves, one grid node for the maps).
# Bytes count every array the kernel must touch once; flops count the
# kernel's FP64 arithmetic per unit (fma = 2).
KERNELS = ["gather B", "curve solve B", "curve->grid map B", "gather G", "curve solve G",
           "curve->grid map G"]
#   gathers (unit = curve node): cell 4 + corner weights 32 + grid value 8 + node value out 8 B;
#                  1 mul + 3 fma = 7 flop
#   curve solve B (unit = curve unknown): load row 8 + rhs rows 24 + factors cp, vp, lp 24 +
#                  v 8 + u 8 B (load and rhs rows carry the row factor ip); rhs 6 (3 fma) +
#                  elimination 2 + upward 2 + back 4 flop (the new values come out of the
#                  solve: no update)
#   curve solve G: rhs coefficient 8 + factors 24 + v 8 + u 8 B; rhs 4 (add, fma, mul) +
#                  elimination 2 + upward 2 + back 4 flop
#   maps (unit = grid node): crossings 16 + coefficients 64 + type 1 + out 8 (+ u_j 8 for
#         the norms) B, 8 fma (+ 1 add and 2 fma for the norms)
BYTES_PER_UNIT = [52.0, 72.0, 81.0, 52.0, 48.0, 89.0]
FLOPS_PER_UNIT = [7.0, 14.0, 16.0, 7.0, 12.0, 21.0]
# The same for the direct curve-to-curve transfer (--transfer direct), whose
# curve solves read the state at their own nodes and whose transfers replace
# the maps (unit = one target curve node):
#   curve solve B: load row 8 + rhs rows 24 + factors 24 + v 8 + u 8 B; rhs 6 +
#                  elimination 2 + upward 2 + back 4 flop
#   curve solve G: rhs coefficient 8 + factors 24 + v 8 + u 8 B; rhs 4 + 2 + 2 + 4 flop
#   transfers: two segment indices 8 + four coefficients 32 + source value 8 + out 8
#              (+ previous state 8 for the norms) B; 1 mul + 3 fma (+ 1 add, 2 fma) flop
KERNELS_DIRECT = ["(none)", "curve solve B (node state)", "transfer B->G", "(none)",
                  "curve solve G (node state)", "transfer G->B + norms"]
BYTES_PER_UNIT_DIRECT = [0.0, 72.0, 56.0, 0.0, 48.0, 64.0]
FLOPS_PER_UNIT_DIRECT = [0.0, 14.0, 7.0, 0.0, 12.0, 12.0]
# DRAM bytes per launch (read + write) of each kernel in the bench's launch
# shape, from one ncu capture of the 2048^2 sheared workload; None where the
# kernel has changed since the capture
NCU_TRAFFIC_SHEARED2048 = [204.3e6, 350.9e6, 398.9e6, 215.5e6, 262.4e6, 435.3e6]
NCU_TRAFFIC_DIRECT_SHEARED2048 = [None, 351.2e6, 235.3e6, None, 263.1e6, 258.9e6]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", "--grid-n", dest="n", type=int, default=2048)
    ap.add_argument("--prec", default="fp64", choices=["fp64", "fp32"])
    ap.add_argument("--tol", type=float, default=1e-8)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--stabilize", type=int, default=0, choices=[0, 1],
                    help="1: SUPG on the B curves (FP64 only)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--anderson", type=int, default=0,
                    help="Anderson extrapolation depth of the stationary iteration (0 = none)")
    ap.add_argument("--transfer", default="grid", choices=["grid", "direct"],
                    help="values between the curve families through the grid (the paper's "
                         "section 6) or directly through the curves' crossings")
    ap.add_argument("--no-direct", action="store_true",
                    help="skip the direct-transfer solve of the same workload in the default line")
    ap.add_argument("--no-oracle", action="store_true",
                    help="skip the oracle's converged solve (the err_vs_oracle figures)")
    ap.add_argument("--other-prec", action=argparse.BooleanOptionalAction, default=True)
    ap.add_argument("--workload", default="sheared",
                    choices=["sheared", "batch", "learned", "data2d", "parabolic", "manufactured",
                             "kernels", "anderson"])
    ap.add_argument("--time-steps", type=int, default=200, help="parabolic workload: time steps")
    ap.add_argument("--count", type=int, default=256)
    # learned warm start: training set, held-out set, Adam steps, minibatch
    ap.add_argument("--train", type=int, default=2048)
    ap.add_argument("--hold", type=int, default=128)
    ap.add_argument("--train-steps", type=int, default=3000)
    ap.add_argument("--batch-size", type=int, default=32)
    return ap.parse_args()


def peaks():
    try:
        with open(PEAKS_FILE) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


class Clocks:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,utilization.gpu,"
              "clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

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
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 10:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None

        def num(x):
            try:
                return float(x)
            except ValueError:
                return float("nan")
        load = [r for r in rows if num(r[4]) >= 50] or rows
        sm = [num(r[1]) for r in load]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in load:
            for k, name in enumerate(names):
                if r[6 + k].lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": num(rows[0][2]),
                "reasons": sorted(reasons), "samples": len(rows), "samples_under_load": len(load)}


def dist_setup(args):
    import torch
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(ws, value, device):
    if ws == 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(ws, value, device):
    if ws == 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def job_rate(ws, ms, units, device):
    """Whole-job throughput of weak-scaled replicas: the units all ranks
    processed over the slowest rank's time.  Returns (ms_max, units_all, rate/s)."""
    ms_max = max_over_ranks(ws, ms, device)
    units_all = sum_over_ranks(ws, units, device)
    return ms_max, units_all, units_all / (ms_max / 1e3)


# ------------------------------------------------------------- oracle legs

def _oracle_converged(n, tol, path, transfer=0, anderson=0):
    """Child process: the oracle's converged stationary solve of the n^2
    sheared workload from u = 0 (the same Δt and tol as the GPU), saved as
    path (.npy) with its step count beside it (.json)."""
    from oracle import oracle as O
    from paper_2411_11041_gb300 import workloads as W
    t0 = time.perf_counter()
    o = O.Oracle(W.sheared(n=n), transfer=transfer, anderson=anderson)
    out, _, it, rel, st = o.solve_stationary(tol=tol, max_iter=200000)
    np.save(path, out)
    with open(path + ".json", "w") as fh:
        json.dump({"iters": it, "status": st, "secs": time.perf_counter() - t0}, fh)


class OracleJob:
    """The oracle's converged solve in a spawned process (one host core), so
    that every result of the run can be compared with it."""

    def __init__(self, n, tol, transfer=0, anderson=0):
        import multiprocessing as mp
        fd, self.path = tempfile.mkstemp(suffix=".npy")
        os.close(fd)
        self.proc = mp.get_context("spawn").Process(target=_oracle_converged,
                                                    args=(n, tol, self.path, transfer, anderson),
                                                    daemon=True)
        self.proc.start()

    def result(self, timeout_s):
        """(u, info) or (None, reason)."""
        self.proc.join(timeout_s)
        if self.proc.is_alive():
            self.proc.terminate()
            return None, f"the oracle had not finished after {timeout_s:.0f} s more"
        try:
            u = np.load(self.path)
            with open(self.path + ".json") as fh:
                info = json.load(fh)
        except (OSError, ValueError) as e:
            return None, f"oracle failed: {e}"
        finally:
            for q in (self.path, self.path + ".json"):
                if os.path.exists(q):
                    os.unlink(q)
        return u, info


def rel_err(u_gpu, u_ref):
    """max |u - u_oracle| / max |u_oracle| over the grid."""
    return float(np.abs(u_gpu - u_ref).max() / max(np.abs(u_ref).max(), 1e-300))


def oracle_sample(n, budget_s=12.0, min_steps=1, transfer=0):
    """Time split steps of the FP64 CPU oracle on the same workload (setup
    excluded) for about budget_s seconds.  Returns (line-DOF/s, steps, secs)."""
    from oracle import oracle as O
    from paper_2411_11041_gb300 import workloads as W
    prob = W.sheared(n=n)
    o = O.Oracle(prob, transfer=transfer)
    unknowns = 0
    for fam in (0, 1):
        off = o.lines(fam)["off"]
        unknowns += int(np.maximum(np.diff(off) - 2, 0).sum())
    dt = o.default_dt()
    u = np.zeros((n, n))
    steps, t0 = 0, time.perf_counter()
    while steps < min_steps or time.perf_counter() - t0 < budget_s:
        _, u = o.split_step(0.5, dt, u)
        steps += 1
    secs = time.perf_counter() - t0
    return unknowns * steps / secs, steps, secs, unknowns


def run_reference(args):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle import oracle as O
    from paper_2411_11041_gb300 import workloads as W
    prob = W.sheared(n=args.n)
    o = O.Oracle(prob, transfer=int(args.transfer == "direct"))
    unknowns = 0
    for fam in (0, 1):
        off = o.lines(fam)["off"]
        unknowns += int(np.maximum(np.diff(off) - 2, 0).sum())
    dt = o.default_dt()
    u = np.zeros((args.n, args.n))
    for _ in range(args.warmup):
        _, u = o.split_step(0.5, dt, u)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        _, u = o.split_step(0.5, dt, u)
    secs = time.perf_counter() - t0
    val = unknowns * args.steps / secs
    sample = (f"{args.steps} split steps (one B and one G sweep each) of the {args.n}^2 "
              "sheared problem per timed run, setup excluded; a full solve takes the "
              "same per-step work times the iteration count")
    line = {
        "impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": secs / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": f"sheared{args.n}", "nodes": args.n * args.n,
                                        "transfer": args.transfer,
                                        "step": "one split step (oracle sample)"},
        "cpu_baseline": {"value": val, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- our leg

def run_ours(args):
    import torch

    from paper_2411_11041_gb300 import ADR_FP32_REFINE, ADR_FP64, Solver
    from paper_2411_11041_gb300 import workloads as W
    ws, rank, local = dist_setup(args)
    direct = args.transfer == "direct"
    job = OracleJob(args.n, args.tol, int(direct), args.anderson) \
        if rank == 0 and not args.no_oracle else None
    # the same workload with the direct transfer and with the accelerated
    # iteration, reported beside the main line (each against its own oracle solve)
    also = not direct and not args.no_direct and ws == 1 and args.prec == "fp64" \
        and not args.stabilize and not args.anderson
    variants = [("direct_transfer", 1, 0)] if also else []
    vjobs = {name: OracleJob(args.n, args.tol, tr, m) for name, tr, m in variants} \
        if not args.no_oracle else {}
    dev = torch.device(f"cuda:{local}")
    torch.cuda.set_device(dev)
    prec = ADR_FP64 if args.prec == "fp64" else ADR_FP32_REFINE
    prob = W.sheared(n=args.n)
    solver = Solver(prob, device=dev, tol=args.tol, max_iter=200000, prec=prec,
                    stabilize=args.stabilize, transfer=int(direct), anderson=args.anderson)
    tuned = solver.autotune(10)  # launch shapes by measurement (adr_autotune), before timing
    unknowns = solver.line_unknowns()
    stream = torch.cuda.current_stream(dev)
    for _ in range(args.warmup):
        solver.solve_stationary()
    torch.cuda.synchronize(dev)
    barrier(ws)
    torch.cuda.synchronize(dev)
    clocks = Clocks(local)
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    iters, dofs, status = [], 0.0, []
    e0.record(stream)
    for _ in range(args.steps):
        u, _, st, code = solver.solve_stationary()
        iters.append(st["iters"])
        dofs += st["line_dofs"]
        status.append(code)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    barrier(ws)
    torch.cuda.synchronize(dev)
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    ms_max, dofs_all, value = job_rate(ws, ms, dofs, dev)
    # per-kernel device time in the solve's launch configuration (CUDA events)
    roof = kernel_roofline(solver, prob, unknowns, direct)
    names = KERNELS_DIRECT if direct else KERNELS
    traffic = NCU_TRAFFIC_DIRECT_SHEARED2048 if direct else NCU_TRAFFIC_SHEARED2048
    k = names.index(roof["kernel"])
    if args.n == 2048 and prec == ADR_FP64 and traffic[k] is not None:
        roof["traffic"] = traffic[k]
        roof["traffic_source"] = "ncu dram__bytes_read.sum + dram__bytes_write.sum, one capture"
        roof["algorithmic_bytes"] = roof["algorithmic_bytes_per_launch"]
    if args.n == 2048 and prec == ADR_FP64 and all(t is not None for t, m in
                                                   zip(traffic, roof["all_kernels_ms_list"]) if m > 0):
        roof["split_step"] = step_hbm(roof, traffic)
    # per split step: B solve, B map / transfer, G solve, G map / transfer, check;
    # per solve: state reset, output (and the initial gather / midpoint of the direct transfer)
    # per split step: (gather,) solve, map or transfer for each family, the check;
    # the gathers are passes of their own in FP64 through the grid; + the
    # extrapolation's 3 kernels
    per_step = (5 if direct else 7) + (3 if args.anderson else 0)
    launches = int(sum(per_step * it + (5 if direct else 3) for it in iters))
    # the other precision mode on the same workload (the direct transfer: the
    # transfer through the grid instead): time to tol and agreement
    other = {}
    if args.other_prec and not args.stabilize and not args.anderson:  # FP32+refine: no SUPG, no extrapolation
        oprec = ADR_FP32_REFINE if prec == ADR_FP64 and not direct else ADR_FP64
        s2 = Solver(prob, device=dev, tol=args.tol, max_iter=200000, prec=oprec)
        s2.solve_stationary()
        torch.cuda.synchronize(dev)
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        reps, it2, d2 = 3, [], 0.0
        for _ in range(reps):
            u2, _, st2, _ = s2.solve_stationary()
            it2.append(st2["iters"])
            d2 += st2["line_dofs"]
        f1.record(stream)
        torch.cuda.synchronize(dev)
        ms2 = f0.elapsed_time(f1)
        diff = float((u2 - u).abs().max() / u.abs().max())
        u_other = u2.cpu().numpy()
        other = {"prec": "fp32+refine" if oprec == ADR_FP32_REFINE else "fp64",
                 "transfer": "grid",
                 "ms_per_step": ms2 / reps, "value": d2 / (ms2 / 1e3), "iters_per_solve": it2,
                 "kernels_ms": dict(zip(KERNELS, s2.time_kernels(reps=20))),
                 "max_rel_diff_vs_this_mode": diff}
        s2.close()
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64" if prec == ADR_FP64 else "f32+f64",
        "data": "synthetic",
        "config": {"workload": f"sheared{args.n}", "nodes": prob.nx * prob.ny,
                   "mu": prob.mu, "sigma": prob.sigma, "tol": args.tol, "prec": args.prec,
                   "stabilize": args.stabilize, "transfer": args.transfer, "anderson": args.anderson,
                   "line_unknowns_per_step": unknowns, "iters_per_solve": iters,
                   "step": "one stationary solve to tol from u=0",
                   "l2": "working set > 129 MB L2 (curve data and maps ~1 GB)",
                   "launch_shape": {"rows_per_thread": tuned[0], "map_blocks_per_sm": tuned[1],
                                    "tuned_ms_per_split_step": tuned[2]},
                   "parallelism": f"replicas x{ws}"},
        "roofline": roof, "gpu_launches": launches, "clocks": clk,
    }
    if other:
        line["other_precision"] = other
    for name, tr, m in variants:
        line[name] = variant_leg(args, prob, dev, stream, tr, m)
    if not args.no_e2e:
        line["e2e"] = e2e(args, prob, dev, prec)
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        v, nst, secs, unk = oracle_sample(args.n, transfer=int(direct))
        line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": f"{nst} split steps of the {args.n}^2 sheared problem "
                                          f"({secs:.1f} s, setup excluded), single thread"}
    if job is not None:
        # every result against the oracle's converged solve (same Δt and tol)
        ref, info = job.result(timeout_s=600)
        if ref is None:
            line["err_vs_oracle"] = {"value": None, "why": info}
        else:
            ev = {"measure": "max |u - u_oracle| / max |u_oracle| over the grid",
                  "oracle_iters": info["iters"], "oracle_secs": info["secs"],
                  args.prec: rel_err(u.cpu().numpy(), ref)}
            if other and not direct:
                ev["fp32+refine" if other["prec"] == "fp32+refine" else "fp64"] = rel_err(u_other, ref)
            ev["tolerance"] = {"fp64": 1e-12, "fp32+refine": 1e-5}
            line["err_vs_oracle"] = ev
    for name, tr, m in variants:
        dl = line[name]
        if name in vjobs:
            ref, info = vjobs[name].result(timeout_s=600)
            if ref is None:
                dl["err_vs_oracle"] = {"value": None, "why": info}
            else:
                dl["err_vs_oracle"] = {"fp64": rel_err(dl["_u"], ref), "oracle_iters": info["iters"],
                                       "oracle_secs": info["secs"], "tolerance": 1e-12,
                                       "oracle": "the oracle's converged solve with the same options"}
        dl.pop("_u", None)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def variant_leg(args, prob, dev, stream, transfer, anderson, reps=3):
    """The same stationary solve with the direct curve-to-curve transfer
    (opts.transfer = 1) and/or the accelerated iteration (opts.anderson),
    FP64: time to tol, iterations, per-kernel roofline."""
    import torch

    from paper_2411_11041_gb300 import Solver
    direct = bool(transfer)
    s = Solver(prob, device=dev, tol=args.tol, max_iter=200000, transfer=transfer, anderson=anderson)
    tuned = s.autotune(10)
    s.solve_stationary()
    torch.cuda.synchronize(dev)
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    its, dofs = [], 0.0
    for _ in range(reps):
        u, _, st, _ = s.solve_stationary()
        its.append(st["iters"])
        dofs += st["line_dofs"]
    f1.record(stream)
    torch.cuda.synchronize(dev)
    ms = f0.elapsed_time(f1)
    unknowns = s.line_unknowns()
    roof = kernel_roofline(s, prob, unknowns, direct)
    names = KERNELS_DIRECT if direct else KERNELS
    traffic = NCU_TRAFFIC_DIRECT_SHEARED2048 if direct else NCU_TRAFFIC_SHEARED2048
    k = names.index(roof["kernel"])
    if args.n == 2048 and traffic[k] is not None:
        roof["traffic"] = traffic[k]
        roof["traffic_source"] = "ncu dram__bytes_read.sum + dram__bytes_write.sum, one capture"
    if args.n == 2048 and all(t is not None for t, m in zip(traffic, roof["all_kernels_ms_list"]) if m > 0):
        roof["split_step"] = step_hbm(roof, traffic)
    out = {"transfer": "direct" if direct else "grid", "anderson": anderson,
           "ms_per_step": ms / reps, "value": dofs / (ms / 1e3), "unit": UNIT,
           "iters_per_solve": its,
           "launch_shape": {"rows_per_thread": tuned[0], "tuned_ms_per_split_step": tuned[2]},
           "roofline": roof, "_u": u.cpu().numpy()}
    s.close()
    return out


def e2e(args, prob, dev, prec):
    """Public-API end to end: pinned host inputs -> device, adr_create,
    adr_solve_stationary, result -> host, every step."""
    import torch

    from paper_2411_11041_gb300 import Solver
    pin = {k: torch.from_numpy(np.ascontiguousarray(getattr(prob, k))).pin_memory()
           for k in ("mask", "beta1", "beta2", "f")}
    h2d = sum(t.numel() * t.element_size() for t in pin.values())
    d2h = prob.nx * prob.ny * 8
    host_out = torch.empty((prob.ny, prob.nx), dtype=torch.float64).pin_memory()

    class P:
        pass

    def one():
        q = P()
        q.nx, q.ny, q.x0, q.y0, q.x1, q.y1 = prob.nx, prob.ny, prob.x0, prob.y0, prob.x1, prob.y1
        q.mu, q.sigma = prob.mu, prob.sigma
        for k, t in pin.items():
            setattr(q, k, t.to(dev, non_blocking=True))
        s = Solver(q, device=dev, tol=args.tol, max_iter=200000, prec=prec,
                   transfer=int(args.transfer == "direct"), anderson=args.anderson)
        u, _, st, _ = s.solve_stationary()
        host_out.copy_(u)
        s.close()
        return st["line_dofs"]

    one()
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    dofs = 0.0
    for _ in range(args.steps):
        dofs += one()
    torch.cuda.synchronize(dev)
    secs = time.perf_counter() - t0
    return {"value": dofs / secs, "unit": UNIT, "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": d2h, "ms_per_step": secs / args.steps * 1e3,
            "includes": "H2D of mask/beta/f from pinned memory, adr_create (geometry setup), "
                        "adr_solve_stationary, D2H of u"}


def run_batch(args):
    """Many problems of uneven size and shape (N ~ U{128..1024}, square /
    disc / L masks, constant flow of random direction): all solved to tol as
    one batch, against the same problems solved one after another."""
    import torch

    from paper_2411_11041_gb300 import ADR_FP32_REFINE, ADR_FP64, Batch, Solver
    from paper_2411_11041_gb300 import partition as PT
    from paper_2411_11041_gb300 import workloads as W
    ws, rank, local = dist_setup(args)
    dev = torch.device(f"cuda:{local}")
    torch.cuda.set_device(dev)
    prec = ADR_FP64 if args.prec == "fp64" else ADR_FP32_REFINE
    allp = W.batch(count=args.count)
    # the problems are independent: each rank solves its own share (LPT on the
    # estimated work), no exchange step
    parts, loads = PT.lpt_split([PT.work_estimate(p) for p in allp], ws)
    probs = [allp[i] for i in parts[rank]]
    t0 = time.perf_counter()
    solvers = [Solver(p, device=dev, tol=args.tol, max_iter=200000, prec=prec, interp_weights=1,
                      anderson=args.anderson)
               for p in probs]
    setup_s = time.perf_counter() - t0
    batch = Batch(solvers)
    t0 = time.perf_counter()
    tuned_rows, tuned_ms = batch.autotune(reps=5)  # rows per thread by measurement, before timing
    tune_s = time.perf_counter() - t0
    stream = torch.cuda.current_stream(dev)
    for _ in range(args.warmup):
        batch.solve()
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier(ws)
    torch.cuda.synchronize(dev)
    e0.record(stream)
    dofs = 0.0
    for _ in range(args.steps):
        outs, stats, st = batch.solve()
        dofs += sum(x["line_dofs"] for x in stats)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    barrier(ws)
    ms_rank = e0.elapsed_time(e1) / args.steps
    ms_batch, dofs_all, _ = job_rate(ws, ms_rank, dofs / args.steps, dev)
    iters = [x["iters"] for x in stats]
    # one problem at a time through its own graph (the same options)
    def one_by_one(ss):
        for s in ss[:4]:
            s.solve_stationary()
        torch.cuda.synchronize(dev)
        e0.record(stream)
        its = []
        for s in ss:
            its.append(s.solve_stationary()[2]["iters"])
        e1.record(stream)
        torch.cuda.synchronize(dev)
        return max_over_ranks(ws, e0.elapsed_time(e1), dev), its
    ms_plain, _ = one_by_one(solvers)
    # where the batch's time goes: the same batch without its slowest tenth
    order = np.argsort(iters)[::-1]
    cut = max(1, len(order) // 10)
    rest = Batch([solvers[i] for i in sorted(order[cut:])]) if len(order) > cut else None
    tail = {}
    if rest is not None:
        rest.solve()
        torch.cuda.synchronize(dev)
        e0.record(stream)
        rest.solve()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms_rest = e0.elapsed_time(e1)
        tail = {"slowest_tenth": cut, "batch_without_slowest_tenth_ms": ms_rest,
                "slowest_tenth_share": 1.0 - ms_rest / ms_batch,
                "active_problems_at_step": {str(k): int(sum(1 for x in iters if x > k))
                                            for k in (0, 50, 100, 150, 200, 300, 500, 800)}}
    # the paper's iteration one by one (no extrapolation), when the batch extrapolates
    unaccel = {}
    if args.anderson:
        plain_solvers = [Solver(p, device=dev, tol=args.tol, max_iter=200000, prec=prec, interp_weights=1)
                         for p in probs]
        ms_unacc, its_unacc = one_by_one(plain_solvers)
        unaccel = {"plain_unaccelerated_sequential_ms": ms_unacc,
                   "unaccelerated_iters_min_median_max": [min(its_unacc), int(np.median(its_unacc)),
                                                          max(its_unacc)],
                   "speedup_vs_unaccelerated_sequential": ms_unacc / ms_batch}
        for s in plain_solvers:
            s.close()
    line = {"metric": METRIC, "value": dofs_all / (ms_batch / 1e3), "unit": UNIT,
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_batch,
            "higher_is_better": True, "scaling": "strong", "vs_baseline": None,
            "dtype": "f64" if prec == ADR_FP64 else "f32+f64", "data": "synthetic",
            "config": {"workload": f"batch{args.count}", "nodes": int(sum(p.nx * p.ny for p in allp)),
                       "tol": args.tol, "iters_min_median_max": [min(iters), int(np.median(iters)), max(iters)],
                       "step": "all problems solved to tol as one batch",
                       "parallelism": f"problems split over {ws} rank(s), LPT on estimated work",
                       "estimated_load_per_rank": loads},
            "plain_sequential_ms": ms_plain, "batched_speedup": ms_plain / ms_batch,
            "setup_s": setup_s, "tail": tail,
            "autotune": {"rows_per_thread": tuned_rows, "ms_per_batched_split_step": tuned_ms,
                         "tune_s": tune_s}}
    line["config"]["anderson"] = args.anderson
    line.update(unaccel)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


# FP32-accumulated BF16 work of the warm-start network per sample (one 64 x 64
# map): 2 * 4096 pixels * 9 taps * sum of Cin * Cout over the eight layers
CNN_FLOPS_FWD = 2 * 4096 * 9 * (24 * 64 + 64 * 64 + 64 * 128 + 2 * 128 * 128 + 128 * 64
                                 + 64 * 64 + 64 * 16)


def bf16_peak():
    try:
        with open(PEAKS_FILE) as fh:
            d = json.load(fh)
        return float(d["bf16_tflops"]), float(d["bf16_tflops_sustained"]), "measured"
    except Exception:
        return 1900.0, 1700.0, "fallback"


def run_learned(args):
    """Learned warm start on 256 x 256 squares: the network is trained on the
    GPU on solutions the batched solver generates, then held-out problems are
    solved to tol from its initial states (network time included), batched.
    Compared with the same batch from u = 0 and with the plain method (one
    problem after another from u = 0)."""
    import torch

    from paper_2411_11041_gb300 import ADR_OK, Batch, Network, Solver
    from paper_2411_11041_gb300 import warmstart as WS
    from paper_2411_11041_gb300 import workloads as W
    dev = torch.device("cuda:0")
    stream = torch.cuda.current_stream(dev)
    t0 = time.perf_counter()
    train = W.learned(args.train, n=256)
    hold = W.learned(args.hold, n=256, seed=W.SEED_BASE + 5)
    draw_s = time.perf_counter() - t0
    net = Network(max(args.batch_size, min(args.hold, 512)))
    # a twentieth of the training problems (at least 64) is kept out of the
    # training to calibrate the gate: the classes where the correction helps
    n_val = max(64, len(train) // 20) if len(train) >= 256 else 0
    val, train = train[len(train) - n_val:], train[:len(train) - n_val]
    t0 = time.perf_counter()
    data = WS.generate(net, train, tol=args.tol, anderson=3)  # the same fixed points, sooner
    torch.cuda.synchronize(dev)
    gen_s = time.perf_counter() - t0
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    losses = WS.train(net, data, args.train_steps, batch=args.batch_size, log_every=500)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    train_ms = e0.elapsed_time(e1)
    step_ms = train_ms / args.train_steps
    gate = WS.calibrate_gate(net, val, tol=args.tol, anderson=args.anderson) if n_val else {}
    hd = WS.generate(net, hold, tol=args.tol, anderson=3)
    zero_loss = 0.5 * float((hd.t.double() ** 2).mean())
    held_loss = net.loss_grad(hd.x[:args.batch_size].contiguous(),
                              hd.t[:args.batch_size].contiguous())[0]
    # forward of (up to 512 of) the held-out set: the tensor-core kernels alone
    n_fwd = min(len(hold), 512)
    x = hd.x[:n_fwd].contiguous()
    for _ in range(3):
        net.forward(x)
    e0.record(stream)
    for _ in range(10):
        net.forward(x)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    fwd_ms = e0.elapsed_time(e1) / 10
    # the timed region: features + network + unpack + batched solve.  The
    # held-out set is solved in batches of at most 512 problems (each 256^2
    # handle holds some 40 MB of curve data, maps and factors): the times add up
    opts = WS.solver_opts(args.tol, anderson=args.anderson)
    ms_learned = ms_zero = ms_paper = 0.0
    sl, sz, sp = [], [], []
    stl = stz = stp = ADR_OK
    clocks = Clocks(0)
    clocks.start()
    for k in range(0, len(hold), 512):
        part = hold[k:k + 512]
        learned = [Solver(p, device=dev, init=1, **opts) for p in part]
        zero = [Solver(p, device=dev, **opts) for p in part]
        paper = [Solver(p, device=dev, init=2, **opts) for p in part]  # eq. u0stationary
        fields = WS.stack(part, dev)
        use = WS.gate_of(gate, part)
        bl, bz, bp = Batch(learned), Batch(zero), Batch(paper)

        def learned_step():
            return bl.solve(WS.initial_states(net, learned, fields, use))

        for _ in range(args.warmup):
            learned_step()
            bz.solve()
            bp.solve()
        torch.cuda.synchronize(dev)
        e0.record(stream)
        for _ in range(args.steps):
            _, s_l, st_l = learned_step()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms_learned += e0.elapsed_time(e1) / args.steps
        e0.record(stream)
        for _ in range(args.steps):
            _, s_z, st_z = bz.solve()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms_zero += e0.elapsed_time(e1) / args.steps
        e0.record(stream)
        for _ in range(args.steps):
            _, s_p, st_p = bp.solve()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms_paper += e0.elapsed_time(e1) / args.steps
        sl += s_l
        sz += s_z
        sp += s_p
        stl, stz, stp = max(stl, st_l), max(stz, st_z), max(stp, st_p)
        for bb in (bl, bz, bp):
            bb.close()
        for s in learned + zero + paper:
            s.close()
        del fields
    clk = clocks.stop()
    # the plain method: one problem after another from u = 0, in chunks of
    # 256 handles (each handle's own solve keeps a graph and a stream)
    ms_plain = 0.0
    plain_opts = WS.solver_opts(args.tol)
    for k in range(0, len(hold), 256):
        chunk = [Solver(p, device=dev, **plain_opts) for p in hold[k:k + 256]]
        for s in chunk:
            s.solve_stationary()
        torch.cuda.synchronize(dev)
        e0.record(stream)
        for s in chunk:
            s.solve_stationary()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms_plain += e0.elapsed_time(e1)
        for s in chunk:
            s.close()
    if stl != ADR_OK or stz != ADR_OK or stp != ADR_OK:
        raise RuntimeError("a held-out solve did not converge")
    itl = np.array([s["iters"] for s in sl])
    itz = np.array([s["iters"] for s in sz])
    itp = np.array([s["iters"] for s in sp])
    # where the learned start gains or loses against the paper's u0: the
    # iteration ratio by decade of mu and by half of the sigma range
    mus = np.array([p.mu for p in hold])
    sgs = np.array([p.sigma for p in hold])
    by_mu = {}
    for lo in (-4, -3, -2):
        sel = (np.log10(mus) >= lo) & (np.log10(mus) < lo + 1)
        if sel.any():
            by_mu[f"1e{lo}..1e{lo + 1}"] = [int(sel.sum()), float(itl[sel].sum() / itp[sel].sum())]
    by_sigma = {}
    for lo, hi in ((0.0, 1.05), (1.05, 3.0)):
        sel = (sgs >= lo) & (sgs < hi)
        if sel.any():
            by_sigma[f"{lo}..{hi}"] = [int(sel.sum()), float(itl[sel].sum() / itp[sel].sum())]
    peak, peak_sus, kind = bf16_peak()
    fwd_tf = CNN_FLOPS_FWD * n_fwd / (fwd_ms * 1e-3) / 1e12
    train_tf = 3 * CNN_FLOPS_FWD * args.batch_size / (step_ms * 1e-3) / 1e12
    # kernels per timed step: the paper's u0 (4 per problem), features, 8
    # convolutions, one unpack per problem, then per batch iteration 2 curve
    # solves, 2 maps, check, compact, flip
    launches = 5 * len(hold) + 1 + 8 + 7 * int(itl.max())
    line = {
        "metric": "held-out 256^2 problems solved to 1e-8 per second (learned warm start, batched)",
        "value": len(hold) / (ms_learned / 1e3), "unit": "problems/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_learned,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64 solve, bf16 net",
        "data": "synthetic",
        "config": {"workload": f"learned256x{args.hold}", "train_problems": len(train),
                   "calibration_problems": n_val,
                   "gate": {f"1e{k}..1e{k + 1}": bool(v) for k, v in sorted(gate.items())},
                   "network_input": "problem data + the paper's initial state (eq. u0stationary)",
                   "train_steps": args.train_steps, "minibatch": args.batch_size, "tol": args.tol,
                   "anderson": args.anderson,
                   "step": "paper u0 + features + network + initial states + batched solve of the "
                           "held-out set (batches of at most 512 problems)"},
        "iters_mean": {"zero_init": float(itz.mean()), "paper_u0_init": float(itp.mean()),
                       "learned_init": float(itl.mean()),
                       "ratio": float(itl.sum() / itz.sum()),
                       "ratio_vs_paper_u0": float(itl.sum() / itp.sum()),
                       "share_of_problems_improved": float((itl < itz).mean()),
                       "share_improved_vs_paper_u0": float((itl < itp).mean()),
                       "share_worse_than_paper_u0": float((itl > itp).mean()),
                       "learned_over_paper_by_mu": by_mu, "learned_over_paper_by_sigma": by_sigma},
        "ms": {"learned_batched": ms_learned, "zero_batched": ms_zero, "paper_u0_batched": ms_paper,
               "plain_sequential": ms_plain},
        "speedup": {"learned_batched_vs_plain": ms_plain / ms_learned,
                    "learned_vs_zero_batched": ms_zero / ms_learned},
        "training": {"draw_s": draw_s, "generate_s": gen_s, "train_s": train_ms / 1e3,
                     "step_ms": step_ms, "train_tflops": train_tf,
                     "held_out_loss": held_loss, "zero_prediction_loss": zero_loss,
                     "loss_log": losses[-3:]},
        "roofline": {"bound": "tensor", "achieved": fwd_tf, "peak": peak, "unit": "TFLOP/s",
                     "frac": fwd_tf / peak, "traffic": None, "peak_kind": kind + " bf16 burst",
                     "kernel": "network forward (8 BF16 convolutions)", "kernel_ms": fwd_ms,
                     "units_per_launch": n_fwd},
        "gpu_launches": launches, "clocks": clk,
    }
    print(json.dumps(line), flush=True)


def run_data2d(args):
    """The paper's experiment (eq. Data2D) as the paper runs it: 50 Crank-Nicolson
    steps of dt = 0.001 from the state of eq. u0stationary, on n x n nodes
    (default 61).  Latency-bound (the grid fits in L2); timed per solve."""
    import torch

    from paper_2411_11041_gb300 import ADR_INIT_PAPER_U0, Solver
    from paper_2411_11041_gb300 import workloads as W
    n = args.n if args.n != 2048 else 61
    prob = W.data2d(n)
    dev = torch.device("cuda:0")
    s = Solver(prob, device=dev, tol=0.0, max_iter=50, dt=1e-3, init=ADR_INIT_PAPER_U0)
    unknowns = s.line_unknowns()
    stream = torch.cuda.current_stream(dev)
    for _ in range(args.warmup):
        s.solve_stationary()
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    dofs = 0.0
    for _ in range(args.steps):
        _, _, st, _ = s.solve_stationary()
        dofs += st["line_dofs"]
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1) / args.steps
    line = {"metric": METRIC.replace("time-to-1e-8 relative update", "50 steps of eq. Data2D"),
            "value": dofs / args.steps / (ms / 1e3), "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": f"data2d{n}", "nodes": n * n, "line_unknowns_per_step": unknowns,
                       "step": "50 split steps, dt = 0.001, theta = 0.5, from u0stationary",
                       "l2": "fits in L2: a latency case"}}
    if not args.no_cpu_baseline:
        from oracle import oracle as O
        o = O.Oracle(prob)
        t0 = time.perf_counter()
        o.solve_stationary(theta=0.5, dt=1e-3, tol=0.0, max_iter=50, init=2)
        secs = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": dofs / args.steps / secs, "unit": UNIT, "cores": 1,
                                "kind": "oracle", "sample": f"the same 50-step solve ({secs:.2f} s)"}
    print(json.dumps(line), flush=True)


def kernel_units(solver, prob, unknowns, direct=False):
    """Units one launch of each sweep kernel processes (curve nodes for the
    gathers and the transfers' targets, curve unknowns for the solves, grid
    nodes for the maps)."""
    nodes = [int(solver.lines(f)["off"][-1]) for f in (0, 1)]
    if direct:
        return [0, unknowns[0], nodes[1], 0, unknowns[1], nodes[0]]
    return [nodes[0], unknowns[0], prob.nx * prob.ny, nodes[1], unknowns[1], prob.nx * prob.ny]


def kernel_roofline(solver, prob, unknowns, direct=False):
    """Dominant sweep kernel of a solver, timed with CUDA events in the
    solve's launch configuration (adr_time_kernels): the roofline object."""
    kms = solver.time_kernels(reps=20)
    units = kernel_units(solver, prob, unknowns, direct)
    names = KERNELS_DIRECT if direct else KERNELS
    bpu = BYTES_PER_UNIT_DIRECT if direct else BYTES_PER_UNIT
    fpu = FLOPS_PER_UNIT_DIRECT if direct else FLOPS_PER_UNIT
    k = int(np.argmax(kms))
    hbm, hbm_kind = peaks()
    gbs = bpu[k] * units[k] / (kms[k] * 1e-3) / 1e9
    tflops = fpu[k] * units[k] / (kms[k] * 1e-3) / 1e12
    return {"bound": "alu", "achieved": tflops, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
            "frac": tflops / FP64_PEAK_TFLOPS, "traffic": None,
            "peak_kind": "FP64 FMA issue peak derived from 152 SMs x 2 FMA/clk x 2.07 GHz",
            "hbm_frac": gbs / hbm, "kernel": names[k], "kernel_ms": kms[k],
            "units_per_launch": units[k], "algorithmic_bytes_per_launch": bpu[k] * units[k],
            "all_kernels_ms": {nm: kms[i] for i, nm in enumerate(names) if kms[i] > 0},
            "all_kernels_hbm_frac": {nm: bpu[i] * units[i] / (kms[i] * 1e-3) / 1e9 / hbm
                                     for i, nm in enumerate(names) if kms[i] > 0},
            "split_step_ms": float(sum(kms)), "all_kernels_ms_list": [float(x) for x in kms],
            "algorithmic_bytes_list": [bpu[i] * units[i] for i in range(len(kms))]}


def step_hbm(roof, traffic):
    """The whole split step against the HBM peak: the DRAM bytes of every
    sweep kernel (one ncu capture each) and their algorithmic bytes over the
    kernels' CUDA-event times back to back."""
    hbm, hbm_kind = peaks()
    kms = roof["all_kernels_ms_list"]
    ms = float(sum(kms))
    dram = float(sum(t for t, m in zip(traffic, kms) if m > 0))
    alg = float(sum(b for b, m in zip(roof["algorithmic_bytes_list"], kms) if m > 0))
    return {"ms": ms, "dram_bytes": dram, "algorithmic_bytes": alg,
            "dram_gbs": dram / (ms * 1e-3) / 1e9, "dram_frac": dram / (ms * 1e-3) / 1e9 / hbm,
            "algorithmic_frac": alg / (ms * 1e-3) / 1e9 / hbm, "peak_gbs": hbm,
            "peak_kind": "measured copy peak" if hbm_kind == "measured" else "fallback copy peak"}


def run_parabolic(args):
    """The parabolic problem (eq. Parabolic1) on n^2 nodes (1024 by default):
    implicit Euler in time, dt = 1e-3, 200 steps from the Gaussian blob, each
    time slice solved by the splitting iteration to the tolerance (mode 1: the
    slice's reaction sigma + 1/dt and load f + u_n/dt).  One timed step = the
    whole 200-step run."""
    import torch

    from paper_2411_11041_gb300 import ADR_FP32_REFINE, ADR_FP64, ADR_OK, Solver
    from paper_2411_11041_gb300 import workloads as W
    from oracle import oracle as O
    n = args.n if args.n != 2048 else 1024
    dt, nsteps = 1e-3, args.time_steps
    prob = W.parabolic(n=n)
    dev = torch.device("cuda:0")
    prec = ADR_FP64 if args.prec == "fp64" else ADR_FP32_REFINE
    s = Solver(prob, device=dev, tol=args.tol, max_iter=200000, prec=prec, anderson=args.anderson)
    unknowns = s.line_unknowns()
    u0 = torch.tensor(prob.u0, device=dev)
    stream = torch.cuda.current_stream(dev)
    # the first slices, against the oracle's
    n_check = 2
    u = u0.clone()
    s.step_parabolic(u, dt, n_check, 1)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    o = O.Oracle(prob, anderson=args.anderson)
    ref, ref_iters, ost = o.step_parabolic(prob.u0, dt, n_check, 1, tol=args.tol, max_iter=200000)
    oracle_check_s = time.perf_counter() - t0
    err_first = rel_err(u.cpu().numpy(), ref)
    for _ in range(args.warmup):
        u = u0.clone()
        s.step_parabolic(u, dt, nsteps, 1)
    torch.cuda.synchronize(dev)
    clocks = Clocks(0)
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    iters, dofs = [], 0.0
    e0.record(stream)
    for _ in range(args.steps):
        u = u0.clone()
        st, code = s.step_parabolic(u, dt, nsteps, 1)
        if code != ADR_OK:
            raise RuntimeError("a time slice did not reach tol")
        iters.append(st["iters"])
        dofs += st["line_dofs"]
    e1.record(stream)
    torch.cuda.synchronize(dev)
    clk = clocks.stop()
    ms = e0.elapsed_time(e1) / args.steps
    roof = kernel_roofline(s, prob, unknowns)
    line = {"metric": METRIC.replace("time-to-1e-8 relative update",
                                     f"{nsteps} implicit-Euler steps, each slice to {args.tol:g}"),
            "value": dofs / args.steps / (ms / 1e3), "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if prec == ADR_FP64 else "f32+f64", "data": "synthetic",
            "config": {"workload": f"parabolic{n}", "nodes": n * n, "dt": dt, "time_steps": nsteps,
                       "mu": prob.mu, "sigma": prob.sigma, "tol": args.tol, "mode": 1,
                       "anderson": args.anderson,
                       "line_unknowns_per_split_step": unknowns,
                       "split_steps_per_run": iters[-1],
                       "split_steps_per_slice": iters[-1] / nsteps,
                       "ms_per_time_step": ms / nsteps,
                       "step": f"one {nsteps}-step run from the Gaussian blob",
                       "l2": "working set ~250 MB > 129 MB L2"},
            "roofline": roof,
            "gpu_launches": int(iters[-1] * (7 + (3 if args.anderson else 0))
                                + nsteps * 4), "clocks": clk,
            "err_vs_oracle": {"measure": "max |u - u_oracle| / max |u_oracle|",
                              "first_slices": n_check, args.prec: err_first,
                              "oracle_split_steps": ref_iters, "oracle_secs": oracle_check_s}}
    if not args.no_cpu_baseline:
        sig = prob.sigma + 1.0 / dt
        pdt = o.default_dt(sigma=sig)
        uo, steps, t0 = prob.u0.copy(), 0, time.perf_counter()
        while time.perf_counter() - t0 < 10.0:
            _, uo = o.split_step(0.5, pdt, uo, sigma=sig, f_extra=prob.u0, fx_scale=1.0 / dt)
            steps += 1
        secs = time.perf_counter() - t0
        rate = (unknowns[0] + unknowns[1]) * steps / secs
        line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": f"{steps} split steps of a {n}^2 time slice ({secs:.1f} s, "
                                          "setup excluded), single thread; a run takes "
                                          f"{iters[-1]} of them: {iters[-1] / (rate / (unknowns[0] + unknowns[1])):.0f} s "
                                          "extrapolated"}
    print(json.dumps(line), flush=True)


def run_manufactured(args):
    """The manufactured-solution problem on 64^2 nodes (u = sin pi x sin pi y,
    beta = (1, 0.5), mu = 0.1, sigma = 1) solved to a relative update of 1e-10
    in FP64.  Fits in L2: a latency case, timed per solve."""
    import torch

    from paper_2411_11041_gb300 import Solver
    from paper_2411_11041_gb300 import workloads as W
    from oracle import oracle as O
    n = args.n if args.n != 2048 else 64
    tol = 1e-10
    prob = W.manufactured(n=n)
    dev = torch.device("cuda:0")
    s = Solver(prob, device=dev, tol=tol, max_iter=200000, anderson=args.anderson,
               transfer=int(args.transfer == "direct"))
    stream = torch.cuda.current_stream(dev)
    for _ in range(args.warmup):
        s.solve_stationary()
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    dofs = 0.0
    for _ in range(args.steps):
        u, _, st, _ = s.solve_stationary()
        dofs += st["line_dofs"]
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1) / args.steps
    o = O.Oracle(prob, anderson=args.anderson, transfer=int(args.transfer == "direct"))
    t0 = time.perf_counter()
    ref, _, it, _, _ = o.solve_stationary(tol=tol, max_iter=200000)
    secs = time.perf_counter() - t0
    ug = u.cpu().numpy()
    line = {"metric": METRIC.replace("1e-8", "1e-10"),
            "value": dofs / args.steps / (ms / 1e3), "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": f"manufactured{n}", "nodes": n * n, "tol": tol,
                       "anderson": args.anderson, "transfer": args.transfer,
                       "split_steps": st["iters"], "step": "one stationary solve to tol from u=0",
                       "l2": "fits in L2: a latency case"},
            "err_vs_oracle": {"measure": "max |u - u_oracle| / max |u_oracle|", "fp64": rel_err(ug, ref),
                              "oracle_split_steps": it},
            "err_vs_exact": float(np.abs(ug - W.exact_manufactured(n)).max()),
            "cpu_baseline": {"value": dofs / args.steps / secs, "unit": UNIT, "cores": 1,
                             "kind": "oracle", "sample": f"the same solve ({secs:.2f} s)"}}
    print(json.dumps(line), flush=True)


def run_anderson(args):
    """The accelerated stationary iteration (opts.anderson) against the plain
    one on the sheared problem at several sizes, both transfers: split steps
    and time to tol per solve (CUDA events, 3 solves after one warm-up), and
    the largest difference between the two answers (the same fixed point)."""
    import torch

    from paper_2411_11041_gb300 import Solver
    from paper_2411_11041_gb300 import workloads as W
    dev = torch.device("cuda:0")
    stream = torch.cuda.current_stream(dev)
    rows = []
    for n in (257, 513, 1025, 2048):
        prob = W.sheared(n=n)
        for transfer in (0, 1):
            base = None
            for m in (0, 1, 3, 5):
                s = Solver(prob, device=dev, tol=args.tol, max_iter=200000, transfer=transfer, anderson=m)
                s.solve_stationary()
                torch.cuda.synchronize(dev)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                for _ in range(3):
                    u, _, st, code = s.solve_stationary()
                e1.record(stream)
                torch.cuda.synchronize(dev)
                if base is None:
                    base = u
                rows.append({"n": n, "transfer": "direct" if transfer else "grid", "anderson": m,
                             "steps": st["iters"], "ms_per_solve": e0.elapsed_time(e1) / 3,
                             "max_rel_diff_vs_plain": float((u - base).abs().max() / base.abs().max())})
                s.close()
    print(json.dumps({"workload": "anderson_sweep", "problem": "sheared", "tol": args.tol,
                      "rows": rows}), flush=True)


def run_kernels(args):
    """Kernel timing only: the n^2 sheared problem's four sweep kernels,
    args.steps back-to-back launches each in the solve's launch configuration
    (the command the ncu recipes capture)."""
    import torch

    from paper_2411_11041_gb300 import ADR_FP32_REFINE, ADR_FP64, Solver
    from paper_2411_11041_gb300 import workloads as W
    prec = ADR_FP64 if args.prec == "fp64" else ADR_FP32_REFINE
    prob = W.sheared(n=args.n)
    direct = args.transfer == "direct"
    s = Solver(prob, device=torch.device("cuda:0"), tol=args.tol, prec=prec, transfer=int(direct))
    kms = s.time_kernels(reps=args.steps)
    torch.cuda.synchronize()
    unknowns = s.line_unknowns()
    print(json.dumps({"workload": f"sheared{args.n}", "prec": args.prec, "transfer": args.transfer,
                      "launches_per_kernel": args.steps,
                      "kernels_ms": dict(zip(KERNELS_DIRECT if direct else KERNELS, kms)),
                      "units_per_launch": kernel_units(s, prob, unknowns, direct),
                      "line_unknowns": unknowns}),
          flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batch":
        run_batch(args)
    elif args.workload == "learned":
        run_learned(args)
    elif args.workload == "data2d":
        run_data2d(args)
    elif args.workload == "parabolic":
        run_parabolic(args)
    elif args.workload == "manufactured":
        run_manufactured(args)
    elif args.workload == "kernels":
        run_kernels(args)
    elif args.workload == "anderson":
        run_anderson(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
