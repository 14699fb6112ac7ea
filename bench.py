#!/usr/bin/env python3
"""Benchmark of the VIP fractional-step solver on one or more GPUs.

Metric: fractional-step node-updates/s with every Poisson solve converged to a
1e-8 relative residual (nodes x steps / seconds), plus the HBM and FP64 rooflines
of the dominant kernel (the Poisson BiCGSTAB launch).

Workload (default): flow past the bumpy cylinder r = 1 + 0.05 sin 12t + 0.02 sin 31t
in the channel [-8,24]x[-8,8] at h = 1/64 (about 2.1M nodes), Re = 200, dt = h/10,
synthetic (generated) node set and an impulsively started uniform inflow, solved
in the form chosen by measurement (the mixed form: FP32 inner BiCGSTAB and V-cycle
under FP64 refinement, every solve stopped on the FP64 residual) with the learned
warm start (the pressure increment extrapolated in time with a coefficient fitted
on the run's own first solves), the multigrid's cell-grid parity chosen per geometry
by measurement at setup (vip.choose_mg_shifts).  Its working set (several GB) exceeds the
129 MB L2, so no flush is needed between timed steps.

The timed steps run three times from one checkpoint of the state: on the device
(the headline value, no host synchronisation inside), with per-phase CUDA events
(the Poisson launch's duration for the roofline), and end to end through the C
ABI with the state loaded from and read back to pinned host memory every step
(host-clocked; the median of three repeats).
The same steps are then timed in the plain all-FP64 form, and the batch of 64
equilateral cavities in both forms (extra keys; --no-batch skips it).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With N > 1 (under torch.distributed.run) each rank runs an independent replica
of the workload on its own GPU (the single-geometry path has no exchange step);
value = all ranks' node updates / max-over-ranks time ("weak" scaling).
--impl reference times the FP64 CPU oracle on the host cores on a bounded sample
of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import queue
import statistics
import subprocess
import sys
import time
from pathlib import Path

ROOT = Path(__file__).resolve().parent
sys.path.insert(0, str(ROOT))

METRIC = "fractional-step node-updates/s at 1e-8 Poisson residual"
UNIT = "node-updates/s"
PEAKS_FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}
E2E_REPEATS = 3
REF_STEPS = 6


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="bumpy_h64",
                    choices=["bumpy_h64", "cylinder_h32", "cavity_256", "triangles64"])
    ap.add_argument("--precision", choices=["auto", "mixed", "fp64", "mg32"], default="auto",
                    help="form of the Krylov solves; auto: the fastest of the three over two "
                         "steps from the warmed-up state (vip.choose_precision, untimed)")
    ap.add_argument("--no-fp64-compare", action="store_true",
                    help="skip timing the same steps in the plain all-FP64 form")
    ap.add_argument("--no-batch", action="store_true",
                    help="skip the batch of 64 equilateral cavities (extra keys)")
    ap.add_argument("--batch-steps", type=int, default=6)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--warm-start", choices=["previous", "extrap", "learned"], default="extrap",
                    help="initial guess of the pressure-increment solve: the previous "
                         "increment; its temporal extrapolation with the coefficient fitted on "
                         "this run's own solves; or that plus the network trained on them")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the default multigrid parameters (omega 1.0, corr 1.5)")
    ap.add_argument("--mg-shift", choices=["zero", "auto"], default="auto",
                    help="parity of each geometry's first multigrid cell grid: 0, 0, or the "
                         "parity with the fewest Poisson iterations over two steps from the "
                         "initial fields under each of the four (untimed setup)")
    ap.add_argument("--ws-samples", type=int, default=24)
    ap.add_argument("--ws-epochs", type=int, default=20)
    ap.add_argument("--no-developed", action="store_true",
                    help="skip the second timed window after the flow has developed")
    return ap.parse_args()


def make_workload(name):
    import workloads as w
    if name == "bumpy_h64":
        h = 1.0 / 64
        ns = w.channel_body(h, ("sines", 1.0, [(0.05, 12), (0.02, 31)]), Re=200.0, dt=0.1 * h,
                            name="bumpy_h64")
        cfg = {"workload": "bumpy cylinder r=1+0.05sin12t+0.02sin31t in channel "
                           "[-8,24]x[-8,8], h=1/64", "nodes": ns.n, "Re": 200.0, "dt": 0.1 * h}
        return ns, cfg
    if name == "cylinder_h32":
        h = 1.0 / 32
        ns = w.channel_body(h, ("circle", 0.5), Re=100.0, dt=0.2 * h)
        return ns, {"workload": "circular cylinder D=1 in channel [-8,24]x[-8,8], h=1/32",
                    "nodes": ns.n, "Re": 100.0, "dt": 0.2 * h}
    if name == "cavity_256":
        ns = w.cavity(256, Re=1000.0)
        return ns, {"workload": "lid-driven cavity 256x256, Re=1000", "nodes": ns.n,
                    "Re": 1000.0, "dt": ns.dt}
    if name == "triangles64":
        nss = w.triangle_batch(64, seed=20140126)
        return nss, {"workload": "64 equilateral lid-driven cavities, n_edge ~ U{64..512}, "
                                 "Re ~ U[100,1000], seed 20140126, one context",
                     "nodes": int(sum(ns.n for ns in nss)), "geometries": len(nss),
                     "dt": "0.25 h per geometry"}
    raise SystemExit(f"unknown workload {name}")


def cpu_sample(name):
    """The bounded sample of the workload that the CPU oracle is timed on."""
    import workloads as w
    if name == "bumpy_h64":
        h = 1.0 / 64
        ns = w.channel_body(h, ("sines", 1.0, [(0.05, 12), (0.02, 31)]), Re=200.0, dt=0.1 * h,
                            xlim=(-2.0, 3.0), ylim=(-1.5, 1.5))
        return ns, "same body, h, Re and dt on the channel cropped to [-2,3]x[-1.5,1.5]"
    if name == "triangles64":
        ns = min(w.triangle_batch(64, seed=20140126), key=lambda g: g.n)
        return ns, f"the batch's smallest geometry ({ns.name})"
    ns, _ = make_workload(name)
    return ns, "full workload"


def peaks():
    p = ROOT / "MEASURED_PEAKS.json"
    if p.exists():
        d = json.loads(p.read_text())
        return d, "measured"
    return PEAKS_FALLBACK, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id):
        self.p = None
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}",
                                       "--format=csv,noheader,nounits", "-lms", "50",
                                       "-i", str(gpu_id)],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            # the first sample comes after nvidia-smi's start-up; wait for it (it is taken
            # before the timed region and not counted), so that the samples kept cover the
            # timed steps
            self.p.stdout.readline()
        except (OSError, FileNotFoundError):
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            out, _ = self.p.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
            out, _ = self.p.communicate()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, val in zip(names, f[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_init():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws <= 1:
        return 0, 1, 0
    import torch
    import torch.distributed as dist
    rank = int(os.environ["RANK"])
    local = int(os.environ.get("LOCAL_RANK", rank))
    backend = "nccl" if torch.cuda.is_available() else "gloo"
    if backend == "nccl":
        torch.cuda.set_device(local)
    dist.init_process_group(backend)
    return rank, ws, local


def throughput(n_nodes, steps, ws, ms_max):
    """Whole-job node-updates/s: every rank steps its own replica of n_nodes nodes, so
    the job processes n_nodes x steps x ws node updates in the slowest rank's time."""
    return n_nodes * steps * ws / (ms_max / 1e3)


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, ws):
    if ws <= 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def time_oracle(name, steps, warmup=0, keep_state=False):
    """Time the CPU oracle, as it stands, on the bounded sample (node-updates/s); with
    keep_state the final (u, v, p, phi) come back under "_state" (not for the line)."""
    from oracle import vip_oracle as vo
    ns, desc = cpu_sample(name)
    t0 = time.perf_counter()
    fs = vo.FractionalStep(vo.Operators(ns), rtol=1e-8)
    setup = time.perf_counter() - t0
    for _ in range(warmup):
        fs.step()
    t0 = time.perf_counter()
    for _ in range(steps):
        fs.step()
    sec = time.perf_counter() - t0
    iters = [s["it_p"] for s in fs.stats[warmup:]]
    out = {"_state": (fs.u, fs.v, fs.p, fs.phi)} if keep_state else {}
    return out | {"value": ns.n * steps / sec, "unit": UNIT, "cores": 1, "kind": "oracle",
                  "sample": f"{steps} step(s) after {warmup} warm-up step(s) from the impulsive "
                            f"start, {ns.n} nodes ({desc}); FP64 NumPy/SciPy, single thread; setup "
                            f"{setup:.1f}s not timed; Poisson iterations {iters}"}


def _oracle_worker(name, steps, state, barrier, q):
    """One oracle process of the all-cores CPU leg: the one-core leg's sample, continued
    from that leg's final state; the timed steps of all processes start together."""
    from oracle import vip_oracle as vo
    ns, _ = cpu_sample(name)
    fs = vo.FractionalStep(vo.Operators(ns), rtol=1e-8)
    fs.set_state(*state)
    barrier.wait(timeout=600)
    t0 = time.perf_counter()
    for _ in range(steps):
        fs.step()
    q.put((ns.n * steps, t0, time.perf_counter()))


def time_oracle_all_cores(name, steps, procs, state):
    """The host's aggregate oracle throughput: `procs` independent single-threaded
    oracle processes (spawned, so none inherits a CUDA context), each on the bounded
    sample from the same state (u, v, p, phi); node updates of all of them / the span
    from the first timed step's start to the last one's end."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    barrier, q = ctx.Barrier(procs), ctx.Queue()
    ps = [ctx.Process(target=_oracle_worker, args=(name, steps, state, barrier, q)) for _ in range(procs)]
    for p in ps:
        p.start()
    res, deadline = [], time.perf_counter() + 900
    while len(res) < procs:
        try:
            res.append(q.get(timeout=5))
        except queue.Empty:
            if any(p.exitcode not in (None, 0) for p in ps) or time.perf_counter() > deadline:
                for p in ps:  # these processes only
                    if p.is_alive():
                        p.terminate()
                raise RuntimeError("an oracle process of the all-cores leg failed")
    for p in ps:
        p.join(timeout=60)
    upd = sum(r[0] for r in res)
    span = max(r[2] for r in res) - min(r[1] for r in res)
    return {"value": upd / span, "unit": UNIT, "cores": procs, "kind": "oracle",
            "sample": f"{procs} independent single-threaded oracle processes, each {steps} step(s) "
                      f"on the one-core leg's sample from the state where that leg ended; node "
                      f"updates of all / the span of their timed steps"}


def run_reference(args, rank, ws):
    if rank != 0:
        return
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    # the oracle takes ~5 s per step on its sample: at most REF_STEPS timed steps after
    # at most one warm-up step, so that the run ends within a minute or so
    steps, warmup = max(1, min(args.steps, REF_STEPS)), min(args.warmup, 1)
    ref = time_oracle(args.workload, steps, warmup)
    _, cfg = make_workload(args.workload)
    line = {"impl": "reference", "metric": METRIC, "value": ref["value"], "unit": UNIT,
            "n_gpus": args.gpus, "steps": steps, "warmup": warmup,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": cfg,
            "cpu_baseline": {"value": ref["value"], "unit": UNIT, "cores": ref["cores"],
                             "kind": "oracle", "sample": ref["sample"]},
            "e2e": {"value": ref["value"], "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# DRAM bytes per inner iteration of the Poisson launch, from one ncu capture of the
# same workload, form and kernel (dram__bytes_read.sum + dram__bytes_write.sum of one
# launch divided by its inner iterations; profiles/): every iteration streams the same
# operator and vectors, so a launch's traffic scales with its iterations.  Keyed by
# workload and form; a form whose kernel changed since its capture has no entry.
TRAFFIC_PER_ITER = {
    # 12.172 GB read + 4.557 GB written by the timed step's launch, 40 iterations
    ("bumpy_h64", "mixed"): 16.729e9 / 40,
    # 25.232 GB + 9.361 GB, 38 iterations
    ("bumpy_h64", "fp64"): 34.592e9 / 38,
    # 129.4 MB + 14.3 MB, 23 iterations (the working set fits in L2)
    ("cylinder_h32", "mixed"): 143.6e6 / 23,
}

# FP64 operations per clock per SM of GB300 (two FP64 FMAs), for the ALU roofline;
# 152 SMs at 2070 MHz give 1.26 TFLOP/s, the part's nominal FP64 rate.
FP64_FLOPS_PER_CLK_SM = 4

PREC_BYTES = {"fp64": (8, 8), "mixed": (4, 4), "mg32": (8, 4)}  # Krylov vectors, V-cycle


def poisson_bytes_per_iter(streamed, rows, tb, tm):
    """Algorithmic DRAM bytes of one inner iteration of the multigrid-preconditioned
    BiCGSTAB, Krylov vectors of tb bytes and V-cycle vectors and operators of tm
    bytes (int32 columns):
      * six passes over the fine operator as stored (value + column per streamed
        entry: the stored entries of ordinary slices plus the distinct stencils of
        the uniform slices; vip_operator_layout), two in the Krylov precision and
        the four fine-level applications of the two V-cycles in the V-cycle's, plus
        the FP32 row sum of every row in each FP32 application (differenced rows);
      * the row-sized vector accesses: p update 4 tb + 2 tm, each V-cycle's fine
        level 3 tb + 8.5 tm (residual, restriction, prolongation, smoothing), v 3 tb,
        s 3 tb + 2 tm, t 3 tb, x/r update 6 tb + 16 (the correction, read and
        written, is 8 bytes in every form) -- 48 accesses in the FP64 form;
      * the coarse levels, 188 B per level-1 cell per V-cycle in FP64 (down: b and the
        inverse diagonal, the 9 coefficients of the 3 x 3 stencil core, a quarter
        of b_{l+1}; up: the same plus the parent's correction and y), half in FP32,
        a quarter of a cell per row and 4/3 of it over all levels."""
    ops = 2 * streamed * (tb + 4) + 4 * streamed * (tm + 4)
    ops += rows * 4 * ((2 if tb == 4 else 0) + (4 if tm == 4 else 0))
    vec = rows * (25 * tb + 21 * tm + 16)
    coarse = 2 * 63 * rows * tm / 8
    return ops + vec + coarse


def poisson_flops_per_iter(nnz, rows):
    """Algorithmic floating-point operations of one inner iteration (an FMA counts
    2): six operator applications (2 nnz each); per row 46 in the Krylov and
    fine-level vector updates and dot products (p 6, two V-cycles' fine level 8 each,
    v 4, s 4, t 6, x/r 10) and 32 on the coarse levels (48 per level-1 cell per
    V-cycle: 3 x 3 stencils down and up, smoothing, restriction, correction; a
    quarter of a cell per row, 4/3 over all levels).  The dense coarsest solves are
    added by the caller (coarsest_per_iter).  In the FP64 form all of them are FP64
    operations; the mixed form does them in FP32."""
    return 12 * nnz + 78 * rows


def coarsest_per_iter(entries, tm):
    """Bytes and operations of the dense coarsest solves of one inner iteration:
    each of the two V-cycles reads every entry of the coarsest inverses once and
    multiplies it into one sum (an FMA)."""
    return 2 * tm * entries, 2 * 2 * entries


def poisson_bytes_per_pass(nnz, rows, tb):
    """One FP64 refinement pass: the FP64 residual SpMV, b, x and the five vectors it
    initialises, and the correction x += d."""
    return nnz * 12 + rows * (8 + 8 + 5 * tb) + rows * (8 + 8 + 8)


def timed_steps(ctx, stream, k):
    """Device time (ms) of k steps on the library's stream, CUDA events on that stream."""
    import torch
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    ctx.vip_step(k)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1)


def form_run(vip, ctx, stream, ckpt, k, prec, ws_mode=None):
    """The k steps after the checkpoint in precision form prec (and warm-start mode
    ws_mode, if given): ms, Poisson inner iterations and refinement passes per step,
    last relative residual, status."""
    ctx.vip_set_solver(prec, 1e-8, 50000, vip.VIP_IDENTITY_EXACT)
    if ws_mode is not None:
        ctx.vip_ws_enable(ws_mode)
    ctx.vip_checkpoint(False, ckpt)
    ctx.vip_step(1)  # captures this form's step graph outside the timed region
    ctx.vip_checkpoint(False, ckpt)
    s0 = ctx.vip_get_stats()
    ms = timed_steps(ctx, stream, k)
    s1 = ctx.vip_get_stats()
    return {"ms_per_step": ms / k,
            "poisson_iters_per_step": (s1.total_poisson_iters - s0.total_poisson_iters) / k,
            "poisson_outer_per_step": (s1.total_poisson_outer - s0.total_poisson_outer) / k,
            "last_poisson_relres": s1.poisson_relres, "status": s1.status}


# Steps from the impulsive start before the second, developed-flow window.
DEVELOP_STEPS = 200


def developed_window(vip, ctx, stream, ckpt, prec, ws_mode, args, N, ws):
    """The timed measurement again, later in the flow: from the checkpoint of the first
    window, untimed steps until DEVELOP_STEPS steps have passed since the impulsive
    start, the warm start refitted on the solves just before (as for the first
    window), two untimed steps, then the same number of timed steps (CUDA events on
    the library's stream, max over ranks)."""
    start = args.warmup + (args.ws_samples + 2 if ws_mode else 0)
    ctx.vip_set_solver(prec, 1e-8, 50000, vip.VIP_IDENTITY_EXACT)
    ctx.vip_ws_enable(0)
    ctx.vip_checkpoint(False, ckpt)
    ctx.vip_step(max(0, DEVELOP_STEPS - start))
    out = {}
    if ws_mode:
        ctx.vip_ws_collect(True, args.ws_samples)
        ctx.vip_step(args.ws_samples)
        ctx.vip_ws_collect(False)
        tc = ctx.vip_ws_train(epochs=args.ws_epochs if ws_mode == 1 else 1, lr=1e-3, seed=7)
        ctx.vip_ws_enable(ws_mode)
        out["extrapolation_coefficient"] = tc.extrap
    ctx.vip_step(2)
    first = max(DEVELOP_STEPS, start) + (args.ws_samples if ws_mode else 0) + 2
    s0 = ctx.vip_get_stats()
    barrier(ws)
    ms = timed_steps(ctx, stream, args.steps)
    barrier(ws)
    ms = max_over_ranks(ms, ws)
    s1 = ctx.vip_get_stats()
    out.update({"window": f"steps {first + 1}-{first + args.steps} from the impulsive start",
                "value": N * args.steps * ws / (ms / 1e3), "unit": UNIT,
                "ms_per_step": ms / args.steps,
                "poisson_iters_per_step": (s1.total_poisson_iters - s0.total_poisson_iters) / args.steps,
                "last_poisson_relres": s1.poisson_relres, "status": s1.status})
    return out


def ALL_FORMS(vip):
    return (vip.VIP_PREC_MIXED, vip.VIP_PREC_FP64, vip.VIP_PREC_MG32)


def batch_lines(vip, dev, stream, steps, prec):
    """The batch of 64 equilateral cavities (one context, each geometry's multigrid
    cell-grid parity chosen, multigrid parameters tuned; untimed setup) in the given
    form and in the plain FP64 form, over the same steps from one checkpoint."""
    nss, cfg = make_workload("triangles64")
    N = int(sum(g.n for g in nss))
    t0 = time.perf_counter()
    shifts, _ = vip.choose_mg_shifts(nss, steps=2, precision=prec, rtol=1e-8, max_iters=50000,
                                     device=dev, stream=stream.cuda_stream)
    ctx = vip.solver_for(nss, precision=prec, rtol=1e-8, max_iters=50000, device=dev,
                         stream=stream.cuda_stream, mg_shifts=shifts)
    tune = vip.autotune(ctx, nss)
    ctx.vip_step(3)
    best, table = vip.choose_precision(ctx, ALL_FORMS(vip))
    ckpt = ctx.vip_checkpoint(True)
    setup = time.perf_counter() - t0
    out = {"workload": cfg["workload"], "nodes": N, "geometries": len(nss), "steps": steps,
           "setup_s": round(setup, 1), "multigrid": {"omega": tune["omega"], "corr": tune["corr"]},
           "chosen_form": vip.PREC_NAMES[best], "form_trials": table}
    for name, p in (("chosen", best), ("fp64", vip.VIP_PREC_FP64)):
        r = form_run(vip, ctx, stream, ckpt, steps, p)
        r["node_updates_per_s"] = N / (r["ms_per_step"] / 1e3)
        out[name] = r
    ctx.close()
    return out


def main():
    args = parse()
    rank, ws, local = dist_init()
    if args.impl == "reference":
        run_reference(args, rank, ws)
        return
    import numpy as np
    import torch

    import paper_1401_6513_gb300 as pkg
    pkg.build()
    vip = pkg.load()
    dev = local
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    ns, cfg = make_workload(args.workload)
    nss = ns if isinstance(ns, list) else [ns]
    PREC = {"mixed": vip.VIP_PREC_MIXED, "fp64": vip.VIP_PREC_FP64, "mg32": vip.VIP_PREC_MG32,
            "auto": vip.VIP_PREC_MIXED}
    prec = PREC[args.precision]
    t0 = time.perf_counter()
    shifts = None
    if args.mg_shift == "auto":
        shifts, _ = vip.choose_mg_shifts(nss, steps=2, precision=prec, rtol=1e-8, max_iters=50000,
                                         device=dev, stream=stream.cuda_stream)
    ctx = vip.solver_for(nss, precision=prec, rtol=1e-8, max_iters=50000, device=dev,
                         stream=stream.cuda_stream, mg_shifts=shifts)
    setup_s = time.perf_counter() - t0
    N = int(sum(g.n for g in nss))
    # multigrid parameters tuned on this workload (untimed; back to the initial fields)
    tune = vip.autotune(ctx, nss) if not args.no_autotune else None
    ctx.vip_step(args.warmup)
    ws_info = None
    ws_mode = {"previous": 0, "learned": 1, "extrap": 2}[args.warm_start]
    if ws_mode:
        # collect solved increments, fit the extrapolation and train the network, then
        # use the guess (untimed)
        t1 = time.perf_counter()
        ctx.vip_ws_collect(True, args.ws_samples)
        ctx.vip_step(args.ws_samples)
        ctx.vip_ws_collect(False)
        tc = ctx.vip_ws_train(epochs=args.ws_epochs if ws_mode == 1 else 1, lr=1e-3, seed=7)
        ctx.vip_ws_enable(ws_mode)
        ctx.vip_step(2)
        ws_info = {"guess": args.warm_start, "samples": args.ws_samples,
                   "epochs": args.ws_epochs if ws_mode == 1 else 1, "extrapolation_coefficient": tc.extrap,
                   "first_loss": tc.first_loss, "final_loss": tc.final_loss, "base_loss": tc.base_loss,
                   "network_kept": bool(tc.net_kept), "collect_train_s": round(time.perf_counter() - t1, 2)}
    form_trials = None
    if args.precision == "auto":
        prec, form_trials = vip.choose_precision(ctx, ALL_FORMS(vip))
    form = vip.PREC_NAMES[prec]
    tb, tm = PREC_BYTES[form]
    torch.cuda.synchronize()
    ckpt = ctx.vip_checkpoint(True)
    # ---- timed region: K steps, device time by CUDA events on the library's stream
    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        uuid = str(dev)
    s0 = ctx.vip_get_stats()
    g0_iters = ctx.vip_get_geometry_iters()
    clocks = Clocks(uuid)
    barrier(ws)
    ms = timed_steps(ctx, stream, args.steps)
    barrier(ws)
    clk = clocks.stop()
    s1 = ctx.vip_get_stats()
    g_iters = ctx.vip_get_geometry_iters() - g0_iters
    ms_max = max_over_ranks(ms, ws)
    value = throughput(N, args.steps, ws, ms_max)
    it_p = s1.total_poisson_iters - s0.total_poisson_iters
    out_p = s1.total_poisson_outer - s0.total_poisson_outer
    it_h = s1.total_helm_iters - s0.total_helm_iters
    # ---- the same steps again with per-phase events (the Poisson launch's duration)
    ctx.vip_checkpoint(False, ckpt)
    ctx.vip_set_profiling(True)
    sp0 = ctx.vip_get_stats()
    ctx.vip_step(args.steps)
    torch.cuda.synchronize()
    ctx.vip_set_profiling(False)
    prof, nprof = ctx.vip_get_profile()
    sp1 = ctx.vip_get_stats()
    it_prof = sp1.total_poisson_iters - sp0.total_poisson_iters
    # ---- roofline of the Poisson BiCGSTAB launch (one per step)
    ptr, _, _ = ctx.vip_get_stencil("POISSON")
    nnz_p = int(ptr[-1])
    rows_p = int(ptr.size - 1)
    lay = ctx.vip_operator_layout("POISSON")
    _, cinv_entries = ctx.vip_multigrid_info()
    # entries one operator pass streams, per real entry (exact for one geometry; a
    # batch's geometries are assigned the table's ratio)
    stream_ratio = (lay["other_entries"] + lay["uniform_entries"]) / max(nnz_p, 1)
    # per geometry: a converged system stops iterating inside the shared launch, so the
    # algorithmic bytes are summed over geometries with their own iteration counts
    bytes_p, flops_p, off, kb = 0, 0, 0, 0
    for gi, g in enumerate(nss):
        nnz_g = int(ptr[off + g.n] - ptr[off])
        rows_g = g.n
        if g.n + off <= N and not np.any(g.kind == vip.VIP_NODE_OUTLET):  # closed: bordered row
            nnz_g += int(ptr[N + kb + 1] - ptr[N + kb])
            rows_g += 1
            kb += 1
        bytes_p += int(g_iters[gi]) * poisson_bytes_per_iter(nnz_g * stream_ratio, rows_g, tb, tm)
        flops_p += int(g_iters[gi]) * poisson_flops_per_iter(nnz_g, rows_g)
        off += g.n
    # dense coarsest solves: every geometry's inverse is read while the launch
    # iterates (an overcount for a batch whose systems finish early; there the
    # inverses are small)
    cb, cf = coarsest_per_iter(cinv_entries, tm)
    bytes_p += it_p * cb
    flops_p += it_p * cf
    fp64_flops = flops_p if form == "fp64" else 0
    bytes_p += out_p * poisson_bytes_per_pass(nnz_p, rows_p, tb)
    fp64_flops += out_p * (2 * nnz_p + 8 * rows_p)  # refinement: residual, 3 dots, x update
    t_pois = prof["poisson"] / 1e3
    tpi = TRAFFIC_PER_ITER.get((args.workload, form))
    traffic = tpi * it_p / max(args.steps, 1) if tpi else None  # per launch (one per step)
    pk, pk_src = peaks()
    hbm = float(pk.get("hbm_gbs", PEAKS_FALLBACK["hbm_gbs"]))
    achieved = bytes_p / t_pois / 1e9 if t_pois > 0 else 0.0
    sm_mhz = float(pk.get("sm_max_mhz", 2070.0))
    fp64_peak = FP64_FLOPS_PER_CLK_SM * torch.cuda.get_device_properties(0).multi_processor_count \
        * sm_mhz * 1e6 / 1e12
    fp64_achieved = fp64_flops / t_pois / 1e12 if t_pois > 0 else 0.0
    roof_hbm = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                "frac": achieved / hbm, "peak_source": f"hbm_gbs {pk_src}",
                "bytes_per_step": bytes_p / max(args.steps, 1)}
    roof_alu = {"bound": "alu", "achieved": fp64_achieved, "peak": fp64_peak, "unit": "TFLOP/s",
                "frac": fp64_achieved / fp64_peak,
                "peak_source": f"FP64: {FP64_FLOPS_PER_CLK_SM} flops/clk/SM x SMs x sm_max_mhz "
                               f"{sm_mhz:.0f} ({pk_src})",
                "fp64_flops_per_step": fp64_flops / max(args.steps, 1)}
    # the binding roof is the one the kernel is closest to; the other is reported beside it
    if roof_alu["frac"] > roof_hbm["frac"]:
        roof, roof_other = roof_alu, roof_hbm
    else:
        roof, roof_other = roof_hbm, roof_alu
    kname = {"mixed": "k_bicgstab<float,float>", "fp64": "k_bicgstab<double,double>",
             "mg32": "k_bicgstab<double,float>"}[form]
    roof = dict(roof, traffic=traffic, kernel=kname + " (Poisson)", operator_layout=lay,
                launch_ms_per_step=t_pois * 1e3 / max(nprof, 1))
    # ---- end to end through the C ABI with pinned host buffers, the same steps: every
    # step loads the state from host memory, steps, and reads the new state back into
    # host memory, from which the next step starts
    bufs = [tuple(torch.empty(N, dtype=torch.float64).pin_memory() for _ in range(3))
            for _ in range(2)]
    oph = torch.empty(N, dtype=torch.float64).pin_memory()
    # host-clocked, so three repeats of the same steps (each from the checkpoint, the
    # pinned buffers refilled from it) and their median, against a stray host stall
    e2e_runs, it_e2e = [], None
    for rep in range(E2E_REPEATS):
        ctx.vip_checkpoint(False, ckpt)
        ctx.vip_get_state(*bufs[0], oph)
        se0 = ctx.vip_get_stats()
        torch.cuda.synchronize()
        barrier(ws)
        t0 = time.perf_counter()
        for k in range(args.steps):
            hu, hv, hp = bufs[k % 2]
            ou, ov, op = bufs[(k + 1) % 2]
            ctx.vip_load_state(hu, hv, hp)
            ctx.vip_step(1)
            ctx.vip_get_state(ou, ov, op, oph)
        dt = time.perf_counter() - t0
        barrier(ws)
        e2e_runs.append(max_over_ranks(dt, ws))
        se1 = ctx.vip_get_stats()
        its = se1.total_poisson_iters - se0.total_poisson_iters
        it_e2e = its if it_e2e in (None, its) else -1  # -1: the repeats differed
    e2e_s = statistics.median(e2e_runs)
    st = se1
    # ---- the plain all-FP64 form on the same steps (same context, multigrid, checkpoint)
    fp64_cmp = prev_cmp = None
    if (form != "fp64" or ws_mode) and not args.no_fp64_compare:
        # the plain all-FP64 form: FP64 solves started from the previous increment
        fp64_cmp = form_run(vip, ctx, stream, ckpt, args.steps, vip.VIP_PREC_FP64, ws_mode=0)
        fp64_cmp["node_updates_per_s"] = N / (fp64_cmp["ms_per_step"] / 1e3)
        fp64_cmp["chosen_over_fp64"] = value / ws / fp64_cmp["node_updates_per_s"]
    if ws_mode and not args.no_fp64_compare:
        # the chosen precision with the previous-increment guess: the warm start's gain
        prev_cmp = form_run(vip, ctx, stream, ckpt, args.steps, prec, ws_mode=0)
        prev_cmp["node_updates_per_s"] = N / (prev_cmp["ms_per_step"] / 1e3)
        prev_cmp["chosen_over_previous_guess"] = value / ws / prev_cmp["node_updates_per_s"]
    developed = None
    if not args.no_developed:
        developed = developed_window(vip, ctx, stream, ckpt, prec, ws_mode, args, N, ws)
    ctx.close()
    batch = None
    if ws == 1 and not args.no_batch and args.workload != "triangles64":
        batch = batch_lines(vip, dev, stream, args.batch_steps, prec)
    if rank != 0:
        return
    cpu = cpu_all = None
    if ws == 1 and not args.no_cpu_baseline:
        # one BLAS thread per oracle process (inherited by the spawned ones)
        os.environ.setdefault("OMP_NUM_THREADS", "1")
        os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")
        cpu = time_oracle(args.workload, 2, 1, keep_state=True)
        state = cpu.pop("_state")
        ncores = min(os.cpu_count() or 1, 16)
        if ncores > 1:
            try:
                cpu_all = time_oracle_all_cores(args.workload, 2, ncores, state)
            except RuntimeError as e:
                cpu_all = {"unavailable": str(e)}
    cfg.update({"global_batch": len(nss), "parallelism": f"replicas x{ws}", "precision": form,
                "precision_choice": ({"by": "measurement (vip.choose_precision, 2 steps each)",
                                      "trials": form_trials} if form_trials else "fixed by --precision"),
                "l2": "working set > L2 (no flush needed)", "setup_s": round(setup_s, 2),
                "poisson_iters_per_step": it_p / max(args.steps, 1),
                "poisson_outer_per_step": out_p / max(args.steps, 1),
                "helmholtz_iters_per_step": it_h / max(args.steps, 1),
                "phase_ms_per_step": {k: round(v / max(nprof, 1), 3) for k, v in prof.items()},
                "same_steps_iters": {"timed": it_p, "profiled": it_prof, "e2e": it_e2e},
                "last_poisson_relres": st.poisson_relres, "status": st.status,
                "warm_start": ws_info or {"guess": "previous increment"},
                "multigrid": tune or {"omega": 1.0, "corr": 1.5, "autotuned": False},
                "mg_cell_shift": ("per geometry, chosen: " + " ".join(
                    f"{sx}{sy}" for sx, sy in shifts)) if shifts else "0 0 (all geometries)"})
    dtype = {"mixed": "f32 inner / f64 residual", "fp64": "f64", "mg32": "f64 Krylov / f32 V-cycle"}
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": dtype[form],
            "data": "synthetic", "config": cfg,
            "roofline": roof,
            "roofline_other": roof_other,
            "e2e": {"value": N * args.steps * ws / e2e_s, "unit": UNIT,
                    "h2d_bytes_per_step": 3 * 8 * N, "d2h_bytes_per_step": 4 * 8 * N,
                    "same_steps_as_value": it_e2e == it_p,
                    "repeats_ms_per_step": [round(t * 1e3 / max(args.steps, 1), 3) for t in e2e_runs],
                    "statistic": f"median of {E2E_REPEATS} repeats"},
            # per step: rhs, Helmholtz, divergence, Poisson, stats, projection; the
            # learned guess adds scales, scatter, six convolutions and gather, the
            # extrapolation alone its gather
            "gpu_launches": (6 + {0: 0, 1: 9, 2: 1}[ws_mode]) * args.steps,
            "clocks": clk}
    if developed is not None:
        line["developed_window"] = developed
    if fp64_cmp is not None:
        line["fp64_same_steps"] = fp64_cmp
    if prev_cmp is not None:
        line["previous_guess_same_steps"] = prev_cmp
    if batch is not None:
        line["batch_64_cavities"] = batch
    if cpu is not None:
        line["cpu_baseline"] = cpu
    if cpu_all is not None:
        line["cpu_baseline_all_cores"] = cpu_all
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
