#!/usr/bin/env python3
"""Benchmark of the VIP fractional-step solver on one or more GPUs.

Metric: fractional-step node-updates/s with every Poisson solve converged to a
1e-8 relative residual (nodes x steps / seconds), plus the HBM and FP64 rooflines
of the dominant kernel (the Poisson BiCGSTAB launch).

Workload (default): flow past the bumpy cylinder r = 1 + 0.05 sin 12t + 0.02 sin 31t
in the channel [-8,24]x[-8,8] at h = 1/64 (about 2.1M nodes), Re = 200, dt = h/10,
multigrid-preconditioned FP64 Krylov solves, synthetic (generated) node set and an
impulsively started uniform inflow.  Its working set (several GB) exceeds the
129 MB L2, so no flush is needed between timed steps.

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


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="bumpy_h64",
                    choices=["bumpy_h64", "cylinder_h32", "cavity_256", "triangles64"])
    ap.add_argument("--precision", choices=["mixed", "fp64"], default="fp64")
    ap.add_argument("--e2e-steps", type=int, default=None)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--warm-start", choices=["previous", "learned"], default="previous",
                    help="initial guess of the pressure-increment solve: the previous "
                         "increment, or the network trained on this run's own solves")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the default multigrid parameters (omega 1.0, corr 1.5)")
    ap.add_argument("--mg-shift", choices=["zero", "auto"], default="zero",
                    help="parity of each geometry's first multigrid cell grid: 0, 0, or the "
                         "parity with the fewest Poisson iterations over two steps from the "
                         "initial fields under each of the four (untimed setup)")
    ap.add_argument("--ws-samples", type=int, default=24)
    ap.add_argument("--ws-epochs", type=int, default=20)
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
                                       "--format=csv,noheader,nounits", "-lms", "200",
                                       "-i", str(gpu_id)],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
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


def time_oracle(name, steps, warmup=0):
    """Time the CPU oracle, as it stands, on the bounded sample (node-updates/s)."""
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
    return {"value": ns.n * steps / sec, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{steps} step(s) after {warmup} warm-up step(s) from the impulsive start, "
                      f"{ns.n} nodes ({desc}); FP64 NumPy/SciPy, single thread; setup "
                      f"{setup:.1f}s not timed; Poisson iterations {iters}"}


def run_reference(args, rank, ws):
    if rank != 0:
        return
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    ref = time_oracle(args.workload, max(1, args.steps), args.warmup)
    _, cfg = make_workload(args.workload)
    line = {"impl": "reference", "metric": METRIC, "value": ref["value"], "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": cfg,
            "cpu_baseline": {"value": ref["value"], "unit": UNIT, "cores": ref["cores"],
                             "kind": "oracle", "sample": ref["sample"]},
            "e2e": {"value": ref["value"], "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# DRAM bytes per inner iteration of the Poisson launch, from one ncu capture of the
# same workload and kernel (dram__bytes_read.sum + dram__bytes_write.sum of one launch
# divided by its iterations); every iteration streams the same operator and vectors,
# so a launch's traffic scales with its iterations (profiles/k_bicgstab_poisson_bumpy_h64.md).
# Re-measured whenever the kernel changes.
TRAFFIC_PER_ITER = {("bumpy_h64", "fp64"): 57.911748608e9 / 62.0}

# FP64 operations per clock per SM of GB300 (two FP64 FMAs), for the ALU roofline;
# 152 SMs at 2070 MHz give 1.26 TFLOP/s, the part's nominal FP64 rate.
FP64_FLOPS_PER_CLK_SM = 4


def poisson_bytes_per_iter(streamed, rows, tb):
    """Algorithmic DRAM bytes of one inner iteration of the multigrid-preconditioned
    BiCGSTAB (vectors of tb bytes, int32 columns):
      * six passes over the operator as stored (value + column per streamed entry:
        the stored entries of ordinary slices plus one stencil per slice whose 32
        rows share it; vip_operator_layout): two Krylov SpMVs and the two fine-level
        residuals of each of the two V-cycles;
      * 48 row-sized vector accesses: p update 6, each V-cycle's fine level 11.5
        (residual 3, restriction 1.5, prolongation 3, smoothing 4), v 3, s 5, t 3,
        x/r update 8;
      * the coarse levels, 188 B per level-1 cell per V-cycle (down: b and the
        inverse diagonal, the 9 coefficients of the 3 x 3 stencil core, a quarter
        of b_{l+1}; up: the same plus the parent's correction and y), a quarter of a
        cell per row and 4/3 of it over all levels: 63 B per row per V-cycle."""
    return 6 * streamed * (tb + 4) + 48 * tb * rows + 2 * 63 * rows


def poisson_flops_per_iter(nnz, rows):
    """Algorithmic FP64 operations of one inner iteration (an FMA counts 2): six
    operator applications (2 nnz each); per row 46 in the Krylov and fine-level
    vector updates and dot products (p 6, two V-cycles' fine level 8 each, v 4, s 4,
    t 6, x/r 10) and 32 on the coarse levels (48 per level-1 cell per V-cycle: 3 x 3
    stencils down and up, smoothing, restriction, correction; a quarter of a cell
    per row, 4/3 over all levels).  The dense coarsest solves are added by the
    caller (coarsest_per_iter)."""
    return 12 * nnz + 78 * rows


def coarsest_per_iter(entries):
    """Bytes and FP64 operations of the dense coarsest solves of one inner
    iteration: each of the two V-cycles reads every entry of the coarsest inverses
    once (FP64) and multiplies it into one sum (an FMA)."""
    return 2 * 8 * entries, 2 * 2 * entries


def poisson_bytes_per_pass(nnz, rows, tb):
    """One FP64 refinement pass: the FP64 residual SpMV, b, x and the five vectors it
    initialises, and the correction x += d."""
    return nnz * 12 + rows * (8 + 8 + 5 * tb) + rows * (8 + 8 + tb)


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
    prec = vip.VIP_PREC_MIXED if args.precision == "mixed" else vip.VIP_PREC_FP64
    t0 = time.perf_counter()
    shifts = None
    if args.mg_shift == "auto":
        shifts, _ = vip.choose_mg_shifts(nss, steps=2, precision=prec, rtol=1e-8, max_iters=50000,
                                         device=dev, stream=stream.cuda_stream)
    ctx = vip.solver_for(nss, precision=prec, rtol=1e-8, max_iters=50000, device=dev,
                         stream=stream.cuda_stream, mg_shifts=shifts)
    setup_s = time.perf_counter() - t0
    N = int(sum(g.n for g in nss))
    # multigrid parameters tuned on this workload (one step, then back to the initial
    # fields; untimed)
    tune = vip.autotune(ctx, nss) if not args.no_autotune else None
    ctx.vip_step(args.warmup)
    ws_info = None
    twin = None
    if args.warm_start == "learned":
        # a twin context takes the same steps with the previous-increment guess, so the
        # iteration counts compare step for step at the same residual
        twin = vip.solver_for(nss, precision=prec, rtol=1e-8, max_iters=50000, device=dev,
                              stream=stream.cuda_stream, mg_shifts=shifts)
        if tune:
            twin.vip_set_multigrid(tune["omega"], tune["corr"])
        twin.vip_step(args.warmup + args.ws_samples + 2)
        # collect solved increments, train, then use the network's guess (untimed)
        t1 = time.perf_counter()
        ctx.vip_ws_collect(True, args.ws_samples)
        ctx.vip_step(args.ws_samples)
        ctx.vip_ws_collect(False)
        tc = ctx.vip_ws_train(epochs=args.ws_epochs, lr=1e-3, seed=7)
        ctx.vip_ws_enable(True)
        ctx.vip_step(2)
        ws_info = {"guess": "learned", "samples": args.ws_samples, "epochs": args.ws_epochs,
                   "first_loss": tc.first_loss, "final_loss": tc.final_loss,
                   "collect_train_s": round(time.perf_counter() - t1, 2)}
    torch.cuda.synchronize()
    s0 = ctx.vip_get_stats()
    g0_iters = ctx.vip_get_geometry_iters()
    # ---- timed region: K steps, device time by CUDA events on the library's stream
    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        uuid = str(dev)
    clocks = Clocks(uuid)
    ctx.vip_set_profiling(True)
    barrier(ws)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    ctx.vip_step(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(ws)
    ms = e0.elapsed_time(e1)
    clk = clocks.stop()
    ctx.vip_set_profiling(False)
    prof, nprof = ctx.vip_get_profile()
    s1 = ctx.vip_get_stats()
    if twin is not None:
        t0s = twin.vip_get_stats()
        twin.vip_step(args.steps)
        t1s = twin.vip_get_stats()
        twin.close()
        ws_info["poisson_iters_per_step_previous_guess_same_steps"] = \
            (t1s.total_poisson_iters - t0s.total_poisson_iters) / max(args.steps, 1)
    ms_max = max_over_ranks(ms, ws)
    value = throughput(N, args.steps, ws, ms_max)
    # ---- roofline of the Poisson BiCGSTAB launch (one per step)
    it_p = s1.total_poisson_iters - s0.total_poisson_iters
    out_p = s1.total_poisson_outer - s0.total_poisson_outer
    it_h = s1.total_helm_iters - s0.total_helm_iters
    ptr, _, _ = ctx.vip_get_stencil("POISSON")
    nnz_p = int(ptr[-1])
    rows_p = int(ptr.size - 1)
    tb = 4 if prec == vip.VIP_PREC_MIXED else 8
    lay = ctx.vip_operator_layout("POISSON")
    _, cinv_entries = ctx.vip_multigrid_info()
    # entries one operator pass streams, per real entry (exact for one geometry; a
    # batch's geometries are assigned the table's ratio)
    stream_ratio = (lay["other_entries"] + lay["uniform_entries"]) / max(nnz_p, 1)
    # per geometry: a converged system stops iterating inside the shared launch, so the
    # algorithmic bytes are summed over geometries with their own iteration counts
    g_iters = ctx.vip_get_geometry_iters() - g0_iters
    bytes_p, flops_p, off, kb = 0, 0, 0, 0
    for gi, g in enumerate(nss):
        nnz_g = int(ptr[off + g.n] - ptr[off])
        rows_g = g.n
        if g.n + off <= N and not np.any(g.kind == vip.VIP_NODE_OUTLET):  # closed: bordered row
            nnz_g += int(ptr[N + kb + 1] - ptr[N + kb])
            rows_g += 1
            kb += 1
        bytes_p += int(g_iters[gi]) * poisson_bytes_per_iter(nnz_g * stream_ratio, rows_g, tb)
        flops_p += int(g_iters[gi]) * poisson_flops_per_iter(nnz_g, rows_g)
        off += g.n
    # dense coarsest solves: every geometry's inverse is read while the launch
    # iterates (an overcount for a batch whose systems finish early; there the
    # inverses are small)
    cb, cf = coarsest_per_iter(cinv_entries)
    bytes_p += it_p * cb
    flops_p += it_p * cf
    bytes_p += out_p * poisson_bytes_per_pass(nnz_p, rows_p, tb)
    flops_p += out_p * (2 * nnz_p + 8 * rows_p)  # refinement: residual, 3 dots, x update
    t_pois = prof["poisson"] / 1e3
    tpi = TRAFFIC_PER_ITER.get((args.workload, args.precision))
    traffic = tpi * it_p / max(args.steps, 1) if tpi else None  # per launch (one per step)
    pk, pk_src = peaks()
    hbm = float(pk.get("hbm_gbs", PEAKS_FALLBACK["hbm_gbs"]))
    achieved = bytes_p / t_pois / 1e9 if t_pois > 0 else 0.0
    sm_mhz = float(pk.get("sm_max_mhz", 2070.0))
    fp64_peak = FP64_FLOPS_PER_CLK_SM * torch.cuda.get_device_properties(0).multi_processor_count \
        * sm_mhz * 1e6 / 1e12
    fp64_achieved = flops_p / t_pois / 1e12 if t_pois > 0 else 0.0
    roof_hbm = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                "frac": achieved / hbm, "peak_source": f"hbm_gbs {pk_src}",
                "bytes_per_step": bytes_p / max(args.steps, 1)}
    roof_alu = {"bound": "alu", "achieved": fp64_achieved, "peak": fp64_peak, "unit": "TFLOP/s",
                "frac": fp64_achieved / fp64_peak,
                "peak_source": f"FP64: {FP64_FLOPS_PER_CLK_SM} flops/clk/SM x SMs x sm_max_mhz "
                               f"{sm_mhz:.0f} ({pk_src})",
                "flops_per_step": flops_p / max(args.steps, 1)}
    # the binding roof is the one the kernel is closest to; the other is reported beside it
    if prec == vip.VIP_PREC_FP64 and roof_alu["frac"] > roof_hbm["frac"]:
        roof, roof_other = roof_alu, roof_hbm
    else:
        roof, roof_other = roof_hbm, roof_alu
    roof = dict(roof, traffic=traffic, kernel="k_bicgstab (Poisson)",
                operator_layout=lay)
    # ---- end to end through the C ABI with pinned host buffers: every step loads the
    # state from host memory, steps, and reads the new state back into host memory,
    # from which the next step starts (the integration continues; same work per step)
    k2 = args.e2e_steps or args.steps
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()  # noqa: E731
    u, v, p, phi = ctx.vip_get_state()
    bufs = [(pin(u), pin(v), pin(p)), tuple(torch.empty(N, dtype=torch.float64).pin_memory()
                                            for _ in range(3))]
    oph = torch.empty(N, dtype=torch.float64).pin_memory()
    torch.cuda.synchronize()
    barrier(ws)
    t0 = time.perf_counter()
    for k in range(k2):
        hu, hv, hp = bufs[k % 2]
        ou, ov, op = bufs[(k + 1) % 2]
        ctx.vip_load_state(hu, hv, hp)
        ctx.vip_step(1)
        ctx.vip_get_state(ou, ov, op, oph)
    e2e_s = time.perf_counter() - t0
    barrier(ws)
    e2e_s = max_over_ranks(e2e_s, ws)
    st = ctx.vip_get_stats()
    ctx.close()
    if rank != 0:
        return
    cpu = None
    if ws == 1 and not args.no_cpu_baseline:
        os.environ.setdefault("OMP_NUM_THREADS", "1")
        cpu = time_oracle(args.workload, 1, 0)
    cfg.update({"global_batch": len(nss), "parallelism": f"replicas x{ws}", "precision": args.precision,
                "l2": "working set > L2 (no flush needed)", "setup_s": round(setup_s, 2),
                "poisson_iters_per_step": it_p / max(args.steps, 1),
                "poisson_outer_per_step": out_p / max(args.steps, 1),
                "helmholtz_iters_per_step": it_h / max(args.steps, 1),
                "phase_ms_per_step": {k: round(v / max(nprof, 1), 3) for k, v in prof.items()},
                "last_poisson_relres": st.poisson_relres, "status": st.status,
                "warm_start": ws_info or {"guess": "previous increment"},
                "multigrid": tune or {"omega": 1.0, "corr": 1.5, "autotuned": False},
                "mg_cell_shift": ("per geometry, chosen: " + " ".join(
                    f"{sx}{sy}" for sx, sy in shifts)) if shifts else "0 0 (all geometries)"})
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f32-inner/f64" if args.precision == "mixed" else "f64",
            "data": "synthetic", "config": cfg,
            "roofline": roof,
            "roofline_other": roof_other,
            "e2e": {"value": N * k2 * ws / e2e_s, "unit": UNIT,
                    "h2d_bytes_per_step": 3 * 8 * N, "d2h_bytes_per_step": 4 * 8 * N},
            # per step: rhs, Helmholtz, divergence, Poisson, stats, projection; the
            # learned guess adds scales, scatter, six convolutions and gather
            "gpu_launches": (6 + (9 if ws_info else 0)) * args.steps,
            "clocks": clk}
    if cpu is not None:
        line["cpu_baseline"] = cpu
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
