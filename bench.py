"""Benchmark of the GB300 S_n sweep path (one JSON line on rank 0).

Workload (N=1): 128^3 jittered hexahedra (2,097,152 cells), 288 directions
(6 x 6 product set per octant), 8 right-hand sides, FP32 psi with compensated
phi sums and an FP64 residual, scattering ratio 0.8, lognormal sigma_t.

One step = one pass of the whole hot path over that input: dependency-graph
build (face classification, level peel, cycle lagging, level-major reorder,
work-unit schedule) followed by a source iteration to tol 1e-6 (emission,
sweep, phi reduction, lag update, FP64 residual, every iteration).

metric: cell-angle updates per second = iterations x cells x directions x
right-hand sides / step time.  Inputs are resident in HBM when the timed
region starts; the sweep's psi array (19.3 GB) is far larger than L2, so no
L2 flush is needed between steps.

--impl reference times the FP64 CPU oracle (the reference arm of this
project) on a bounded sample of the same workload on the host cores.
"""

from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "cell-angle updates/s"
UNIT = "cell-angle-rhs updates/s"
WORKLOAD = "hex128_jitter0.15_288dirs_8rhs_fp32_si_tol1e-6"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    p.add_argument("--n", type=int, default=128, help="hex edge (128 = the benchmark workload)")
    p.add_argument("--mode", type=int, default=1, help="1 level-synchronous (CUDA graph), 2 data-driven persistent")
    p.add_argument("--priority", type=int, default=0)
    p.add_argument("--layering", type=int, default=0, help="0 octant-aligned layers, 1 longest-path levels")
    p.add_argument("--cluster", type=int, default=32)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    return p.parse_args()


# ---- multi-process plumbing (replicas: every rank runs its own full problem) ----
def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def aggregate(units: float, ms: float, world: int, backend_device=None):
    """Whole-job throughput: units summed over ranks / the slowest rank's time."""
    if world <= 1:
        return units, ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([units, ms], dtype=torch.float64, device=backend_device)
    u = t[:1].clone()
    m = t[1:].clone()
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    dist.all_reduce(m, op=dist.ReduceOp.MAX)
    return float(u.item()), float(m.item())


# ---- clocks during the timed region ---------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index=0):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
        except (OSError, ValueError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

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
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return None


# ---- the reference arm: FP64 CPU oracle on a bounded sample -----------------------
def oracle_sample(wl, dirs, w, n_dirs_sample, nthreads):
    """Oracle DAG build + one sweep of n_dirs_sample directions of the workload;
    returns (cell-angle-rhs updates, seconds)."""
    import numpy as np

    import oracle

    sample = np.linspace(0, len(dirs) - 1, n_dirs_sample).astype(int)
    src = wl["q"] / (4 * math.pi)
    t0 = time.perf_counter()
    o = oracle.build_dags(wl, dirs[sample])
    o.sweep(wl["sigma_t"], src, w[sample], nthreads=nthreads)
    dt = time.perf_counter() - t0
    return float(n_dirs_sample) * wl["n_cells"] * wl["q"].shape[0], dt


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle
    from inputs import make_workload

    wl = make_workload(3, n=args.n)
    dirs, w = oracle.product_quadrature(*wl["spec"]["quad"])
    nt = oracle.max_threads()
    nd = max(2, min(len(dirs), 4 * nt if args.n >= 128 else len(dirs)))
    for _ in range(args.warmup):
        oracle_sample(wl, dirs, w, nd, nt)
    tot_u, tot_s = 0.0, 0.0
    for _ in range(args.steps):
        u, s = oracle_sample(wl, dirs, w, nd, nt)
        tot_u += u
        tot_s += s
    value = tot_u / tot_s
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_s / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD if args.n == 128 else f"hex{args.n}_288dirs_8rhs"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": nt, "kind": "oracle",
                         "sample": f"per step: oracle DAG build + one sweep of {nd} of 288 directions, "
                                   f"all 8 right-hand sides, full {wl['n_cells']}-cell mesh, {nt} OpenMP threads"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---- the GPU arm ---------------------------------------------------------------------
def run_gpu(args):
    import numpy as np
    import torch

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from inputs import make_workload
    from paper_1803_09876_gb300 import build as libbuild
    from paper_1803_09876_gb300 import jsweep as J

    libbuild.build()
    J.load()
    J.use_torch_allocator()
    wl = make_workload(3, n=args.n)
    N, R = wl["n_cells"], wl["q"].shape[0]
    npol, naz = wl["spec"]["quad"]
    dirs, w = J.jsweep_quadrature_product(npol, naz)
    M = len(dirs)
    mesh = J.mesh_from_dict(wl)
    quad = J.jsweep_quadrature_create(dirs, w)
    opt = J.jsweep_options_default(sweep_mode=args.mode, priority=args.priority, cluster_cells=args.cluster,
                                   layering=args.layering)
    dev = torch.device("cuda", local)
    sig = torch.as_tensor(wl["sigma_t"], dtype=torch.float32, device=dev)
    cr = torch.as_tensor(wl["c_ratio"], dtype=torch.float32, device=dev)
    q = torch.as_tensor(wl["q"], dtype=torch.float32, device=dev).contiguous()
    phi = torch.empty((R, N), dtype=torch.float32, device=dev)
    tol, max_iters = 1e-6, 1000
    stream = torch.cuda.current_stream()

    def step():
        dags = J.jsweep_build_dags(mesh, quad, opt)
        _, it, res, ok = J.jsweep_source_iterate(dags, sig, cr, q, tol=tol, max_iters=max_iters, phi_out=phi)
        return dags, it, res

    for _ in range(args.warmup):
        dags, it, res = step()
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(stream)
    iters, launches, build_ms, sweep_ms, phi_ms = 0, 0, 0.0, [], []
    for _ in range(args.steps):
        dags, it, res = step()
        iters += it
        tm = dags.timing()
        launches += tm["build_launches"] + tm["call_launches"]
        build_ms += tm["build_ms"]
        sweep_ms.append(tm["sweep_ms"])
        phi_ms.append(tm["phi_ms"])
    ev1.record(stream)
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    units = float(iters) * N * M * R
    units_all, ms_all = aggregate(units, ms, ws, dev)
    value = units_all / (ms_all / 1e3)

    # ---- dominant kernel: one sweep (sweep kernel + phi reduction), timed alone
    dags = J.jsweep_build_dags(mesh, quad, opt)
    src = (q / (4 * math.pi)).contiguous()
    reps = 5
    for _ in range(2):
        J.jsweep_sweep(dags, sig, src, phi_out=phi)
    t_sweep, t_phi = [], []
    for _ in range(reps):
        J.jsweep_sweep(dags, sig, src, phi_out=phi)
        tm = dags.timing()
        t_sweep.append(tm["sweep_ms"])
        t_phi.append(tm["phi_ms"])
    sw_ms = statistics.median(t_sweep)
    ph_ms = statistics.median(t_phi)
    # algorithmic bytes per (cell, direction) of one sweep: psi written once and
    # read once (R p each), order index 4 B, incoming mask 1 B, per-cell data
    # G = 128 B (hex) plus sources in and phi out (2 R p) once per sweep, i.e.
    # per direction (G + 2 R p) / M
    p = 4
    G = 128
    B = 2 * R * p + 5 + (G + 2 * R * p) / M
    alg_bytes = B * N * M
    achieved = alg_bytes / ((sw_ms + ph_ms) / 1e3) / 1e9
    peaks = measured_peaks()
    peak = peaks["hbm_gbs"] if peaks else 6800.0
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": None,
            "kernel": ("sweep (level-synchronous CUDA graph)" if args.mode == 1 else "sweep (data-driven persistent)")
                      + " + phi reduction, one sweep of all directions",
            "alg_bytes_per_cell_dir": B, "sweep_ms": sw_ms, "phi_ms": ph_ms,
            "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured)" if peaks else "fallback 6.8 TB/s"}
    sweep_rate = N * M * R / ((sw_ms + ph_ms) / 1e3)

    # ---- end to end through the public API with host buffers
    e2e = None
    if not args.no_e2e:
        h_sig = torch.as_tensor(wl["sigma_t"], dtype=torch.float32).pin_memory()
        h_cr = torch.as_tensor(wl["c_ratio"], dtype=torch.float32).pin_memory()
        h_q = torch.as_tensor(wl["q"], dtype=torch.float32).contiguous().pin_memory()
        h_phi = torch.empty((R, N), dtype=torch.float32).pin_memory()
        d_sig, d_cr, d_q = torch.empty_like(sig), torch.empty_like(cr), torch.empty_like(q)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        it_e2e = 0
        for _ in range(args.steps):
            d_sig.copy_(h_sig, non_blocking=True)
            d_cr.copy_(h_cr, non_blocking=True)
            d_q.copy_(h_q, non_blocking=True)
            dg = J.jsweep_build_dags(mesh, quad, opt)
            _, it, _, _ = J.jsweep_source_iterate(dg, d_sig, d_cr, d_q, tol=tol, max_iters=max_iters, phi_out=phi)
            h_phi.copy_(phi, non_blocking=True)
            it_e2e += it
        e1.record(stream)
        torch.cuda.synchronize()
        e_ms = e0.elapsed_time(e1)
        eu, em = aggregate(float(it_e2e) * N * M * R, e_ms, ws, dev)
        e2e = {"value": eu / (em / 1e3), "unit": UNIT,
               "h2d_bytes_per_step": int(h_sig.numel() * 4 + h_cr.numel() * 4 + h_q.numel() * 4),
               "d2h_bytes_per_step": int(h_phi.numel() * 4)}

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        import oracle
        d64, w64 = oracle.product_quadrature(npol, naz)
        nt = oracle.max_threads()
        nd = max(2, 2 * nt)
        u, s = oracle_sample(wl, d64, w64, nd, nt)
        cpu = {"value": u / s, "unit": UNIT, "cores": nt, "kind": "oracle",
               "sample": f"oracle DAG build + one sweep of {nd} of {M} directions, all {R} right-hand sides, "
                         f"full {N}-cell mesh, {nt} OpenMP threads ({s:.1f} s)"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_all / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD if args.n == 128 else f"hex{args.n}_288dirs_8rhs",
                       "cells": N, "directions": M, "rhs": R, "sweep_mode": args.mode,
                       "priority": args.priority, "cluster_cells": args.cluster, "layering": args.layering,
                       "l2": "inputs larger than L2 (psi 19.3 GB), no flush",
                       "parallelism": f"replicas x{ws}", "si_iterations_per_step": iters / args.steps},
            "roofline": roof,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": launches,
            "clocks": clk,
            "phases_ms": {"dag_build_mean": build_ms / args.steps, "sweep_kernel_median": sw_ms,
                          "phi_reduction_median": ph_ms},
            "sweep_only_rate": sweep_rate,
        }
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
