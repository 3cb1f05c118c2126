#!/usr/bin/env python3
"""Benchmark: grid-point updates per second (GLUPS) of the pressure solve.

One step = one complete solve of the 500^3 Gaussian-blob workload (125 M
cells, FP32 gradients, 20 random blobs, 3 % noise) from P^0 = 0 to
eps_R <= 1e-8: FP32 multigrid-preconditioned conjugate-gradient sweeps on
the fixed-point system inside an FP64 iterative-refinement loop (FP64
residual, norms and constant removal).  value = (valid cells x stencil
applications, every multigrid level counted with its own cells) / device
time, summed over the timed steps (the production plan: each CG segment
one captured CUDA graph that loops on the device until it converges).  Per-kernel times for the roofline come from the same
K solves repeated in profile mode right after (every launch bracketed by
CUDA events).  The same solve without the preconditioner and the same
scheme in FP64 are timed beside it.  Inputs
(1.5 GB of gradients, 1 GB of pressure, ~6 GB of work vectors) are far
larger than L2, so no flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--size n] [--no-e2e] [--no-cpu] [--no-fp64]

--impl reference times the CPU oracle (plain FP64 CG written from the paper)
on this machine's host cores on a bounded sample of the same workload.
Under torchrun (N > 1) every rank solves its own replica (the path has no
exchange step); value sums the ranks' updates over the slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import glob
import json
import os
import re
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "GLUPS (grid-point updates/s) of the solve to tolerance"
TOL = 1e-8


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


TRAFFIC = os.path.join(ROOT, "profiles", "traffic_gaussian_blobs_3d.json")


def _kernel_source_hash():
    from paper_2311_16935_gb300 import profile_traffic

    return profile_traffic.kernel_source_hash()


def _profiled_traffic(kernel: str, cells: int):
    """DRAM bytes per launch of `kernel` (name up to its template arguments)
    from the machine-written ncu summary, scaled to `cells` per launch; None
    when the summary was taken on other kernel sources or lacks the kernel."""
    try:
        with open(TRAFFIC) as fh:
            d = json.load(fh)
    except Exception:
        return None
    if d.get("kernel_source_hash") != _kernel_source_hash():
        return None
    ks = d.get("kernels", {})
    if kernel in ks:  # one instantiation, named with its template arguments
        return ks[kernel]["dram_bytes_per_cell"] * cells
    hits = [v for k, v in ks.items() if k.startswith(kernel + "<")]
    if len(hits) != 1:
        return None
    return hits[0]["dram_bytes_per_cell"] * cells


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = f"/tmp/osmodi_clocks_{os.getpid()}.csv"

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                          "-lms", "200"], stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            for line in open(self.path):
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
        except Exception:
            pass
        sm_sorted = sorted(sm)
        return {"sm_mhz": sm_sorted[len(sm_sorted) // 2] if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _crop_problem(c=100):
    """The c^3 crop at (200, 200, 200) of the 500^3 Gaussian-blob field (same
    blob parameters), FP32 gradients on the host."""
    from paper_2311_16935_gb300 import inputs

    params = inputs.blob_params(20, (500, 500, 500), (5.0, 40.0), 4)
    return inputs.gaussian_blobs_3d(n=(c, c, c), origin=(200, 200, 200), box=(500, 500, 500), params=params,
                                    device="cpu", dtype=torch_float32())


def _host_bytes_available():
    try:
        return os.sysconf("SC_AVPHYS_PAGES") * os.sysconf("SC_PAGE_SIZE")
    except (ValueError, OSError, AttributeError):
        return 0


def _cpu_baseline(grad_full_host=None, gpu_plain_cg_iters=None, size_crop=100, timed_iters=50):
    """The oracle (FP64 CG, as written) on the host cores.

    (1) measured: the 100^3 crop of the same Gaussian-blob field solved to
        eps_R <= 1e-8; value = cells x (iterations + 2) / time, in GLUPS.
    (2) extrapolated: the full 500^3 field, `timed_iters` CG iterations timed
        (the difference of a 1 + timed_iters and a 1-iteration run, so the
        set-up is not counted), times the iteration count of the same
        unpreconditioned CG on the GPU to the same tolerance (the same
        algorithm in exact arithmetic), plus the measured set-up."""
    import numpy as np

    import oracle

    c = size_crop
    prob = _crop_problem(c)
    grid = oracle.Grid(np.ones((c, c, c), bool), (1.0, 1.0, 1.0))
    f = prob.grad.double().numpy()
    t0 = time.perf_counter()
    P, it, res = oracle.solve_cg(grid, f, tol=TOL, maxit=100000)
    dt = time.perf_counter() - t0
    threads = oracle.num_threads()
    out = {"value": grid.n * (it + 2) / dt / 1e9, "unit": "GLUPS", "cores": threads, "kind": "oracle",
           "sample": f"oracle FP64 CG (ray-count operator) on a {c}^3 crop of the 500^3 blob field to eps_R<={TOL}: "
                     f"{it} iterations in {dt:.2f} s",
           "crop_time_to_tolerance_s": dt, "crop_iterations": it}
    if grad_full_host is not None and gpu_plain_cg_iters:
        n3 = grad_full_host.shape[1:]
        cells = int(np.prod(n3))
        # the oracle's ray-count array (14 doubles per cell), gradients, source,
        # pressure and CG vectors: about 200 B per cell
        if _host_bytes_available() < 220 * cells:
            out["full_size"] = {"skipped": f"host memory: {_host_bytes_available() / 1e9:.0f} GB available, "
                                           f"~{220 * cells / 1e9:.0f} GB needed"}
            return out
        gridf = oracle.Grid(np.ones(tuple(n3), bool), (1.0, 1.0, 1.0))
        ff = grad_full_host.double().numpy()
        t0 = time.perf_counter()
        oracle.solve_cg(gridf, ff, tol=TOL, maxit=1)
        t1 = time.perf_counter()
        oracle.solve_cg(gridf, ff, tol=TOL, maxit=1 + timed_iters)
        t2 = time.perf_counter()
        per_it = max((t2 - t1) - (t1 - t0), 1e-9) / timed_iters
        setup = max((t1 - t0) - per_it, 0.0)
        out["full_size"] = {"kind": "extrapolated", "cells": cells, "timed_iterations": timed_iters,
                            "seconds_per_iteration": per_it, "setup_s": setup,
                            "iterations_to_tolerance": int(gpu_plain_cg_iters),
                            "iteration_count_source": "the same unpreconditioned CG on the GPU (this run)",
                            "time_to_tolerance_s": setup + per_it * gpu_plain_cg_iters,
                            "GLUPS": cells * gpu_plain_cg_iters / (setup + per_it * gpu_plain_cg_iters) / 1e9}
    return out


def _cpu_baseline_batched(count, sample=8, tol=1e-10):
    """The oracle (FP64 CG, as written) on the host cores for the batched
    PIV workload: `sample` evenly spaced snapshots of the `count` solved to
    eps_R <= tol one after another, extrapolated to all `count` by the
    sampled time per snapshot."""
    import numpy as np

    import oracle
    from paper_2311_16935_gb300 import inputs

    idx = sorted({int(round(k * (count - 1) / max(sample - 1, 1))) for k in range(sample)})
    secs, its, cells = [], [], []
    for i in idx:
        pr = inputs.piv_snapshot_2d(i, device="cpu")
        grid = oracle.Grid(pr.mask.numpy().astype(bool), pr.spacing)
        f = pr.grad.double().numpy()
        t0 = time.perf_counter()
        _, it, _ = oracle.solve_cg(grid, f, tol=tol, maxit=1_000_000)
        secs.append(time.perf_counter() - t0)
        its.append(int(it))
        cells.append(int(grid.n))
    per = sum(secs) / len(secs)
    return {"kind": "oracle", "cores": oracle.num_threads(), "unit": "solves/s", "value": 1.0 / per,
            "sample": f"oracle FP64 CG to eps_R<={tol} on snapshots {idx} of the {count} (valid cells "
                      f"{min(cells)}-{max(cells)}, {min(its)}-{max(its)} iterations, {sum(secs):.1f} s)",
            "extrapolated_seconds_for_all": per * count, "extrapolation": "mean time per sampled snapshot x count"}


def torch_float32():
    import torch

    return torch.float32


def run_reference(args):
    """--impl reference: the CPU oracle, bounded sample per step."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import numpy as np

    import oracle
    from paper_2311_16935_gb300 import inputs

    c = args.ref_crop
    params = inputs.blob_params(20, (500, 500, 500), (5.0, 40.0), 4)
    prob = inputs.gaussian_blobs_3d(n=(c, c, c), origin=(200, 200, 200), box=(500, 500, 500), params=params,
                                    device="cpu", dtype=torch_float32())
    grid = oracle.Grid(np.ones((c, c, c), bool), (1.0, 1.0, 1.0))
    f = prob.grad.double().numpy()
    for _ in range(args.warmup):
        oracle.solve_cg(grid, f, tol=TOL, maxit=args.ref_iters)
    total_updates, total_t = 0.0, 0.0
    for _ in range(args.steps):
        t0 = time.perf_counter()
        P, it, res = oracle.solve_cg(grid, f, tol=TOL, maxit=args.ref_iters)
        dt = time.perf_counter() - t0
        total_updates += grid.n * (it + 2)
        total_t += dt
    v = total_updates / total_t / 1e9
    sample = (f"oracle FP64 CG on a {c}^3 crop of the 500^3 blob field, {args.ref_iters} iterations per step "
              f"(bounded sample)")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "GLUPS", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_t / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "gaussian_blobs_3d_500^3 (bounded CPU sample)", "crop": c},
            "cpu_baseline": {"value": v, "unit": "GLUPS", "cores": oracle.num_threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": v, "unit": "GLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--size", type=int, default=500)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-cg", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-front", action="store_true")
    ap.add_argument("--no-many", action="store_true")
    ap.add_argument("--streams", type=int, default=8)
    ap.add_argument("--batch-count", type=int, default=512)
    ap.add_argument("--ref-crop", type=int, default=100)
    ap.add_argument("--ref-iters", type=int, default=150)
    ap.add_argument("--cpu-full", type=int, default=1,
                    help="1: also time 50 oracle CG iterations at the full size (extrapolated baseline)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import torch.distributed as dist

    from paper_2311_16935_gb300 import replicas

    info_r = replicas.RankInfo.from_env()
    world, rank, local = info_r.world, info_r.rank, info_r.local
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    group = replicas.RankGroup(info_r, device="cuda")
    barrier, max_over_ranks, sum_over_ranks = group.barrier, group.max, group.sum

    from paper_2311_16935_gb300 import build, inputs

    build.build()
    from paper_2311_16935_gb300 import osmodi as osm

    n = args.size
    prob = inputs.gaussian_blobs_3d(n=(n, n, n), device="cuda", dtype=torch.float32)
    grad = prob.grad
    dims = (n, n, n)
    # the production plan (CG iterations as captured CUDA graphs) for the
    # timed region, and the same plan in profile mode (every kernel of the
    # iterations launched with CUDA events around it) for the per-kernel times
    plan = osm.Plan(3, dims, (1.0, 1.0, 1.0), None, precision=osm.FP32_REFINE, precond=1)
    plan_prof = osm.Plan(3, dims, (1.0, 1.0, 1.0), None, precision=osm.FP32_REFINE, precond=1, profile=1)
    info = plan.info()
    stream = torch.cuda.current_stream()
    p = torch.zeros((n, n, n), dtype=torch.float64, device="cuda")
    plan.workspace()

    for pl in (plan, plan_prof):
        for _ in range(args.warmup):
            p.zero_()
            r = pl.solve(grad, p, TOL)
            assert r.status == osm.OK, r.as_dict()
    torch.cuda.synchronize()

    # timed region: K full solves
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    results = []
    barrier()
    torch.cuda.synchronize()
    with Clocks(local) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            p.zero_()
            r = plan.solve(grad, p, TOL)
            results.append(r.as_dict())
        ev1.record(stream)
        torch.cuda.synchronize()
    barrier()
    # the same K solves in profile mode, right after: per-kernel CUDA events
    # on the solve's stream (the kernels are the timed region's; the events
    # and the uncaptured launches only add gaps between them)
    ka_ms = ka_n = kb_ms = kb_n = mg_ms = mg_n = sw_ms = sw_n = r64_ms = r64_n = 0.0
    pv0, pv1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with Clocks(local) as clk_prof:
        pv0.record(stream)
        for _ in range(args.steps):
            p.zero_()
            r = plan_prof.solve(grad, p, TOL)
            assert r.status == osm.OK, r.as_dict()
            ks = plan_prof.kernel_stats()
            ka_ms += ks["cg_apply_ms"]
            ka_n += ks["cg_apply_launches"]
            kb_ms += ks["cg_update_ms"]
            kb_n += ks["cg_update_launches"]
            mg_ms += ks["precond_ms"]
            mg_n += ks["precond_applications"]
            r64_ms += ks["residual64_ms"]
            r64_n += ks["residual64_launches"]
            km = plan_prof.kernel_stats_precond()
            sw_ms += km["mg_sweep_ms"]
            sw_n += km["mg_sweep_launches"]
        pv1.record(stream)
        torch.cuda.synchronize()
    prof_ms = pv0.elapsed_time(pv1)
    plan_prof.close()
    del plan_prof
    updates = sum(r["point_updates"] for r in results)
    ups, ms_max = replicas.aggregate_throughput(updates, ev0.elapsed_time(ev1), group)
    value = ups / 1e9
    clocks = clk.summary()
    if any(r["status"] != osm.OK for r in results):
        raise SystemExit(f"solve did not converge: {results}")

    # roofline of the dominant kernel: the multigrid fine-level fused
    # red-black sweep (one full sweep per launch: every cell updated once,
    # out of place).  Algorithmic bytes per point update: read z_in, r
    # (2 x 4 B) + code (1 B), write z_out (4 B) = 13 B; updates per launch =
    # the cells of the padded box (padding cells are written too).  Two
    # launches per V-cycle are timed with CUDA events on the solve's stream.
    cells = info["n_box"]
    peak, peak_kind = _peaks()
    sw_avg = sw_ms / max(sw_n, 1)
    per_update = 13.0
    sw_bytes = per_update * cells
    # the timed launches are the plain sweeps (the second pre-sweep and the
    # first post-sweep: no start from zero, no dot product)
    sw_traffic = _profiled_traffic("k_mg_fine_rb_fused<float, 16, 16, 0, 0, 0, 0>", cells)
    # the CG kernel applying the stencil: read z (the preconditioned residual),
    # p_old, x (3 x 4 B) + code (1 B); write p, q, x (3 x 4 B)
    ka_avg = ka_ms / max(ka_n, 1)
    kb_avg = kb_ms / max(kb_n, 1)
    r64_avg = r64_ms / max(r64_n, 1)
    # FP64 refinement residual r = b - L P: bounded by min(HBM, FP64).  Per
    # cell: read P, b (2 x 8 B) + code (1 B), write r (4 B) = 21 B, and 8 FP64
    # instructions (3 neighbour sums; b - D p and the three axis terms as
    # fused multiply-adds; r^2 into the sum): 13 FP64 flops
    try:
        fp64_gflops = osm.probe_fp64()
    except Exception:
        fp64_gflops = None
    res_fp64 = None
    if fp64_gflops and r64_ms > 0:
        inst_rate = fp64_gflops / 2.0 * 1e9          # FP64 FMA instructions/s (one per pipe slot)
        # per cell: 3 adds (axis sums), 5 fma (b - D p, three axis terms,
        # ||r||^2); the FP32 rounding of r runs on the integer units
        t_fp64 = 8.0 * cells / inst_rate              # s per launch at the FP64 instruction peak
        t_hbm = 21.0 * cells / (peak * 1e9)
        res_fp64 = {"fp64_peak_gflops_measured": fp64_gflops, "fp64_instructions_per_cell": 8,
                    "fp64_flops_per_cell": 13, "bound_ms_fp64": t_fp64 * 1e3, "bound_ms_hbm": t_hbm * 1e3,
                    "bound": "fp64" if t_fp64 > t_hbm else "hbm",
                    "frac_of_bound": max(t_fp64, t_hbm) / (r64_avg / 1e3)}

    line = {"metric": METRIC, "value": value, "unit": "GLUPS", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"gaussian_blobs_3d_{n}^3", "cells": n ** 3, "tol_eps_R": TOL,
                       "precision": "fp32 sweeps + fp64 refinement (fp64 residual, norms, mean removal)",
                       "scheme": "multigrid-preconditioned CG on the fixed-point system (two red-black SOR "
                                 "sweeps before and after the coarse correction)",
                       "glups_counting": "valid cells x stencil applications on every level; a red-black "
                                         "half-sweep counts half",
                       "l2": "inputs and work vectors (>5 GB) exceed L2; no flush needed",
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "time_to_tolerance_s": ms_max / args.steps / 1e3,
            "solves_per_s": args.steps * world / (ms_max / 1e3),
            "iterations": {"cg": results[-1]["inner_iters"], "refine_steps": results[-1]["refine_steps"],
                           "eps_R": results[-1]["eps_R"]},
            "roofline": {"bound": "hbm",
                         "kernel": "k_mg_fine_rb_fused (multigrid fine-level red-black sweep, both colours in one pass)",
                         "achieved": sw_bytes / (sw_avg / 1e3) / 1e9, "peak": peak, "unit": "GB/s",
                         "frac": sw_bytes / (sw_avg / 1e3) / 1e9 / peak, "peak_source": peak_kind,
                         "traffic": sw_traffic,
                         "traffic_per_cell": sw_traffic / cells if sw_traffic else None,
                         "algorithmic_bytes_per_update": per_update, "updates_per_launch": cells,
                         "bytes_per_launch": sw_bytes, "avg_launch_ms": sw_avg, "launches_timed": sw_n,
                         "timing": "CUDA events on the solve's stream around every fine-sweep launch of the K "
                                   "profile-mode solves run right after the timed region",
                         "clocks_while_timed": clk_prof.summary(),
                         "other_kernels": [
                             {"name": "k_cg_a (p = z + beta p_old, q = L p, x update, p.q)", "avg_launch_ms": ka_avg,
                              "bytes_per_launch": 25.0 * cells,
                              "achieved": 25.0 * cells / (ka_avg / 1e3) / 1e9 if ka_avg > 0 else None,
                              "traffic": _profiled_traffic("k_cg_a", cells)},
                             {"name": "k_cg_b (r update + r.r)", "avg_launch_ms": kb_avg, "bytes_per_launch": 12.0 * cells,
                              "achieved": 12.0 * cells / (kb_avg / 1e3) / 1e9 if kb_avg > 0 else None,
                              "traffic": _profiled_traffic("k_cg_b", cells)},
                             {"name": "k_residual (r = b - L P in FP64, norms)",
                              "avg_launch_ms": r64_avg, "bytes_per_launch": 21.0 * cells,
                              "achieved": 21.0 * cells / (r64_avg / 1e3) / 1e9 if r64_ms > 0 else None,
                              "traffic": _profiled_traffic("k_residual", cells),
                              "fp64_roofline": res_fp64}]},
            "clocks": clocks, "gpu_launches": int(sum(r["kernel_launches"] for r in results)),
            "preconditioner": {"levels": info.get("mg_levels"), "applications": mg_n,
                               "avg_application_ms": mg_ms / max(mg_n, 1)},
            # where one profiled solve's device time goes (its CUDA events;
            # "rest" = source term, residual starts, CG set-up, folds, output,
            # convergence checks, and the gaps the events add)
            "time_breakdown_ms_per_solve": {
                "timing": "the K solves after the timed region, in profile mode (same kernels, each launch "
                          "bracketed by CUDA events, no graph capture)",
                "profiled_ms_per_solve": prof_ms / args.steps,
                "preconditioner": mg_ms / args.steps, "cg_apply": ka_ms / args.steps,
                "cg_update": kb_ms / args.steps, "refinement_residual": r64_ms / args.steps,
                "refinement_residual_launches": r64_n / args.steps,
                "rest": prof_ms / args.steps - (mg_ms + ka_ms + kb_ms + r64_ms) / args.steps}}

    # the same solve in FP64 arithmetic throughout (same scheme), and the
    # FP32+refinement solve without the preconditioner (time-to-tolerance
    # comparisons on the same GPU)
    def timed_solve(pl):
        p.zero_()
        pl.solve(grad, p, TOL)  # warm-up (graph capture)
        torch.cuda.synchronize()
        p.zero_()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        rr = pl.solve(grad, p, TOL)
        t1.record(stream)
        torch.cuda.synchronize()
        return t0.elapsed_time(t1) / 1e3, rr

    if not args.no_fp64:
        plan64 = osm.Plan(3, dims, (1.0, 1.0, 1.0), None, precision=osm.FP64, precond=1)
        t64, r64 = timed_solve(plan64)
        line["fp64_plain"] = {"scheme": "same (multigrid-preconditioned CG), every vector and operation in FP64",
                              "time_to_tolerance_s": t64, "cg": r64.inner_iters, "eps_R": r64.eps_R,
                              "status": r64.status, "speedup_fp32_refine": t64 / line["time_to_tolerance_s"]}
        plan64.close()
        del plan64
    # the same solve with the refinement loop in float-float arithmetic
    # (options.refine_ff: ~48-bit P, b and residual on the FP32 units instead
    # of FP64); a variant, not the configuration's FP64 residual
    if not args.no_fp64:
        td = line["time_to_tolerance_s"]
        plan_ff = osm.Plan(3, dims, (1.0, 1.0, 1.0), None, precision=osm.FP32_REFINE, precond=1, refine_ff=1)
        tff, rff = timed_solve(plan_ff)
        line["float_float_refinement"] = {"time_to_tolerance_s": tff, "cg": rff.inner_iters, "eps_R": rff.eps_R,
                                          "status": rff.status, "speedup_vs_fp64_refinement": td / tff,
                                          "timing": "one solve, against the timed region's mean"}
        plan_ff.close()
        del plan_ff
    if not args.no_cg:
        plan_cg = osm.Plan(3, dims, (1.0, 1.0, 1.0), None, precision=osm.FP32_REFINE)
        tcg, rcg = timed_solve(plan_cg)
        line["cg_unpreconditioned"] = {"time_to_tolerance_s": tcg, "cg": rcg.inner_iters, "eps_R": rcg.eps_R,
                                       "status": rcg.status, "GLUPS": rcg.point_updates / tcg / 1e9,
                                       "speedup_preconditioned": tcg / line["time_to_tolerance_s"]}
        plan_cg.close()
        del plan_cg

    # the same solve by the V-cycle of one-colour half-sweeps (two passes per
    # red-black sweep on the plan's grid) instead of the fused sweeps
    if not args.no_fp64:
        osm.debug_set(osm.DEBUG_MG_UNFUSED, 1)
        try:
            plan_u = osm.Plan(3, dims, (1.0, 1.0, 1.0), None, precision=osm.FP32_REFINE, precond=1)
            tu, ru = timed_solve(plan_u)
            plan_u.close()
            del plan_u
        finally:
            osm.debug_set(osm.DEBUG_MG_UNFUSED, osm.DEBUG_DEFAULT)
        line["half_sweep_vcycle"] = {"time_to_tolerance_s": tu, "cg": ru.inner_iters, "eps_R": ru.eps_R,
                                     "status": ru.status,
                                     "fused_speedup": tu / line["time_to_tolerance_s"]}

    # the CPU baseline's 100^3 crop of the same field, solved on the GPU by the
    # benchmark's own configuration (time to the same tolerance)
    crop = _crop_problem(100)
    plan_c = osm.Plan(3, (100, 100, 100), (1.0, 1.0, 1.0), None, precision=osm.FP32_REFINE, precond=1)
    gc_dev = crop.grad.cuda()
    pc_dev = torch.zeros((100, 100, 100), dtype=torch.float64, device="cuda")
    plan_c.solve(gc_dev, pc_dev, TOL)  # warm-up
    torch.cuda.synchronize()
    pc_dev.zero_()
    c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    c0.record(stream)
    rc_ = plan_c.solve(gc_dev, pc_dev, TOL)
    c1.record(stream)
    torch.cuda.synchronize()
    line["crop_gpu"] = {"workload": "gaussian_blobs_3d 100^3 crop (the CPU baseline's sample)",
                        "time_to_tolerance_s": c0.elapsed_time(c1) / 1e3, "cg": rc_.inner_iters,
                        "eps_R": rc_.eps_R, "status": rc_.status}
    plan_c.close()
    del plan_c, gc_dev, pc_dev, crop
    grad_host = grad.cpu() if (rank == 0 and world == 1 and not args.no_cpu and args.cpu_full) else None

    # end to end through the C interface with host buffers: the gradient and
    # P^0 live in page-locked host memory and P is returned there; the solve's
    # kernels read and write them directly over the Grace-Blackwell host link
    # (no staging copies), so every transfer happens inside the timed region
    if not args.no_e2e:
        g_host = grad.cpu().pin_memory()
        p_host = torch.empty((n, n, n), dtype=torch.float64).pin_memory()
        # same solve; P^0 = 0 without reading p (p is output only)
        plan_e = osm.Plan(3, dims, (1.0, 1.0, 1.0), None, precision=osm.FP32_REFINE, precond=1, zero_start=1)
        e_updates = 0.0
        r_e = plan_e.solve(g_host, p_host, TOL)  # warm-up on host buffers
        assert r_e.status == osm.OK, r_e.as_dict()
        barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            r_e = plan_e.solve(g_host, p_host, TOL)
            e_updates += r_e.point_updates
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        e_ms = max_over_ranks(e0.elapsed_time(e1))
        line["e2e"] = {"value": sum_over_ranks(e_updates) / (e_ms / 1e3) / 1e9, "unit": "GLUPS",
                       "h2d_bytes_per_step": g_host.numel() * 4,
                       "d2h_bytes_per_step": p_host.numel() * 8,
                       "transfer": "the solve reads the pinned host gradient and writes P into pinned host memory "
                                   "(kernels address host memory over the host link; P^0 = 0 is not read)",
                       "ms_per_step": e_ms / args.steps}
        plan_e.close()
        # the same solves through the staged form of the call, for comparison:
        # the gradient copied into a device buffer and P copied back
        # (cudaMemcpyAsync on the solve's stream, both inside the timed region)
        g_dev = p_dev = plan_s = None
        try:
            g_dev = torch.empty(g_host.shape, dtype=g_host.dtype, device="cuda")
            p_dev = torch.empty((n, n, n), dtype=torch.float64, device="cuda")
            plan_s = osm.Plan(3, dims, (1.0, 1.0, 1.0), None, precision=osm.FP32_REFINE, precond=1, zero_start=1)
            g_dev.copy_(g_host, non_blocking=True)
            r_s = plan_s.solve(g_dev, p_dev, TOL)  # warm-up
            assert r_s.status == osm.OK, r_s.as_dict()
            p_host.copy_(p_dev, non_blocking=True)
            torch.cuda.synchronize()
            s_updates = 0.0
            e0.record(stream)
            for _ in range(args.steps):
                g_dev.copy_(g_host, non_blocking=True)
                r_s = plan_s.solve(g_dev, p_dev, TOL)
                p_host.copy_(p_dev, non_blocking=True)
                s_updates += r_s.point_updates
            e1.record(stream)
            torch.cuda.synchronize()
            s_ms = e0.elapsed_time(e1)
            line["e2e_staged"] = {"value": s_updates / (s_ms / 1e3) / 1e9, "unit": "GLUPS",
                                  "h2d_bytes_per_step": g_host.numel() * 4, "d2h_bytes_per_step": p_host.numel() * 8,
                                  "transfer": "pinned host gradient copied to a device buffer, the solve on device "
                                              "buffers, P copied back to pinned host memory (timed on this rank)",
                                  "ms_per_step": s_ms / args.steps}
        except Exception as exc:  # a comparison, never fatal to the bench line
            line["e2e_staged"] = {"error": repr(exc)[:200]}
        finally:
            if plan_s is not None:
                plan_s.close()
            del g_dev, p_dev, plan_s
        del g_host, p_host, plan_e
    else:
        line["e2e"] = None

    # the source-term front end (Eq. RANS_f) on the same grid: mean velocity
    # and Reynolds stresses in, the gradient field out (inputs > L2)
    if not args.no_front:
        gen = torch.Generator(device="cuda").manual_seed(5)
        U = torch.randn((3, n, n, n), device="cuda", dtype=torch.float32, generator=gen)
        R = 0.1 * torch.randn((6, n, n, n), device="cuda", dtype=torch.float32, generator=gen)
        plan.source_rans(U, R)  # warm-up
        torch.cuda.synchronize()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 3
        f0.record(stream)
        for _ in range(reps):
            out_f = plan.source_rans(U, R)
        f1.record(stream)
        torch.cuda.synchronize()
        f_ms = f0.elapsed_time(f1) / reps
        f_bytes = 52.0 * n ** 3  # read U (12) + stresses (24) + class word (4), write f (12)
        line["front_end"] = {"kernel": "k_front_rans<3> (Eq. RANS_f source from U and stresses)",
                             "ms": f_ms, "bytes_per_launch": f_bytes,
                             "achieved_GBps": f_bytes / (f_ms / 1e3) / 1e9,
                             "frac": f_bytes / (f_ms / 1e3) / 1e9 / peak, "peak_source": peak_kind}
        del U, R, out_f
        torch.cuda.empty_cache()

    # the batched workload: PIV-like snapshots of uneven sizes and masks, one
    # persistent launch per batch with the multigrid V-cycle inside it
    # (reported beside the headline)
    if not args.no_batch:
        del grad, p
        plan.close()
        torch.cuda.empty_cache()
        probs = [inputs.piv_snapshot_2d(i, device="cuda") for i in range(args.batch_count)]
        plans_b = [osm.Plan(2, pr.dims, pr.spacing, pr.mask.cuda(), precond=1) for pr in probs]
        batch = osm.Batch(plans_b)
        grads_b = [pr.grad for pr in probs]
        outs = [torch.zeros(pr.mask.shape, dtype=torch.float64, device="cuda") for pr in probs]
        depth = batch.autotune(grads_b, outs)  # tile depth of the persistent kernel
        graph = batch.capture(grads_b, outs, 1e-10)  # one graph: tables, resets, persistent launch, states
        for o in outs:
            o.zero_()
        graph.launch(stream)  # warm-up replay
        graph.results()
        for o in outs:
            o.zero_()
        torch.cuda.synchronize()
        b0, b1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        b0.record(stream)
        graph.launch(stream)
        b1.record(stream)
        torch.cuda.synchronize()
        st_b, res_b = graph.results()
        bms = b0.elapsed_time(b1)
        graph.close()
        its = [r.inner_iters for r in res_b]
        line["batched_piv"] = {"workload": f"piv_batch_2d_{args.batch_count}", "tol_eps_R": 1e-10,
                               "cells": int(sum(pr.mask.numel() for pr in probs)),
                               "valid_cells": int(sum(int(pr.mask.sum()) for pr in probs)),
                               "status": st_b, "converged": int(sum(r.status == osm.OK for r in res_b)),
                               "seconds": bms / 1e3, "solves_per_s": args.batch_count / (bms / 1e3),
                               "GLUPS": sum(r.point_updates for r in res_b) / (bms / 1e3) / 1e9,
                               "cg_iterations_min_mean_max": [min(its), float(sum(its)) / len(its), max(its)],
                               "launches": 1, "graph_captured": True, "tile_depth_chunks_per_thread": depth,
                               "preconditioner": "multigrid V-cycle (damped Jacobi) inside the persistent launch"}
        # the same launch without the preconditioner (plain CG), for comparison
        plans_p = [osm.Plan(2, pr.dims, pr.spacing, pr.mask.cuda()) for pr in probs]
        batch_p = osm.Batch(plans_p)
        for o in outs:
            o.zero_()
        torch.cuda.synchronize()
        b0.record(stream)
        st_p, res_p = batch_p.solve(grads_b, outs, 1e-10, stream=stream)
        b1.record(stream)
        torch.cuda.synchronize()
        pms = b0.elapsed_time(b1)
        its_p = [r.inner_iters for r in res_p]
        line["batched_piv"]["plain_cg_in_launch"] = {
            "status": st_p, "seconds": pms / 1e3, "solves_per_s": args.batch_count / (pms / 1e3),
            "cg_iterations_min_mean_max": [min(its_p), float(sum(its_p)) / len(its_p), max(its_p)],
            "timer": "CUDA events around one direct (not graph-captured) batched call"}
        del batch_p, plans_p
        # the same snapshots, each solved by the multigrid-preconditioned CG,
        # spread over host threads driving their own streams (osmodi_solve_many)
        if not args.no_many:
            plans_m = [osm.Plan(2, pr.dims, pr.spacing, pr.mask.cuda(), precond=1) for pr in probs]
            many = osm.Many(plans_m, streams=args.streams)
            for o in outs:
                o.zero_()
            many.solve(grads_b, outs, 1e-10)  # warm-up: every plan captures its CUDA graphs
            for o in outs:
                o.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            st_m, res_m = many.solve(grads_b, outs, 1e-10)
            dt_m = time.perf_counter() - t0
            its_m = [r.inner_iters for r in res_m]
            line["batched_piv"]["multistream_multigrid"] = {
                "streams": many.streams, "status": st_m, "converged": int(sum(r.status == osm.OK for r in res_m)),
                "seconds": dt_m, "timer": "host clock around the synchronous call (inputs resident)",
                "solves_per_s": args.batch_count / dt_m,
                "GLUPS": sum(r.point_updates for r in res_m) / dt_m / 1e9,
                "cg_iterations_min_mean_max": [min(its_m), float(sum(its_m)) / len(its_m), max(its_m)],
                "kernel_launches": int(sum(r.kernel_launches for r in res_m))}
            del many, plans_m
        del batch, plans_b, probs, grads_b, outs
    if rank == 0 and world == 1 and not args.no_cpu:
        try:
            cg_its = line.get("cg_unpreconditioned", {}).get("cg")
            line["cpu_baseline"] = _cpu_baseline(grad_host if args.cpu_full else None, cg_its)
            if "batched_piv" in line:
                try:
                    line["batched_piv"]["cpu_baseline"] = _cpu_baseline_batched(args.batch_count)
                except Exception as e:  # reported, never fatal to the bench line
                    line["batched_piv"]["cpu_baseline"] = {"error": repr(e)[:200]}
            if "crop_gpu" in line:
                cb = line["cpu_baseline"]
                line["crop_gpu"]["cpu_oracle_time_to_tolerance_s"] = cb["crop_time_to_tolerance_s"]
                line["crop_gpu"]["speedup_vs_cpu_oracle"] = (cb["crop_time_to_tolerance_s"] /
                                                             line["crop_gpu"]["time_to_tolerance_s"])
        except Exception as exc:  # the baseline is context, never the measurement
            line["cpu_baseline"] = {"error": str(exc)}
    line["kernel_source_hash"] = _kernel_source_hash()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if args.no_batch:
        plan.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
