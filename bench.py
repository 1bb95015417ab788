#!/usr/bin/env python
"""Throughput of the pseudo-particle Exact mapping on one GB300.

A step is one pass of the whole path over the 1e6-particle cloud:
build_tree -> make_pseudo_particles (selection, neighbour search, node h-solver)
-> build_voronoi (262,144 cells) -> find_pairs -> map_exact (mixed FP32/FP64)
-> map_back to the pseudo-particles and the particles.

value = particle-cell pairs mapped per second of step time (all ranks).
Prints one JSON line (rank 0).  `--impl reference` times the FP64 CPU oracle
on a bounded sample of the same workload instead.
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

METRIC = "particle-cell pairs mapped/s (mixed vs FP64) at stated max rel. err; % of roofline"
# name -> (workload, whether the step builds pseudo-particles from a tree)
WORKLOADS = {
    "pseudo_1e6": ("pseudo_1M_particles_262k_cells", True),
    "pseudo_2e5": ("pseudo_200k_particles_52k_cells", True),
    "sphere_1e5": ("sphere_100k_particles_25k_cells", False),
    "batched_64": ("batched_64_snapshots", True),
    "full_8m": ("full_8M_particles_2M_cells", True),
    "direct_8m": ("full_8M_particles_2M_cells_tree_off", False),
}
# workloads whose FP64 reference pass over every pair would take longer than
# the timed steps: accuracy on a random sample of pairs instead
ACCURACY_SAMPLE = {"full_8m": 2_000_000, "direct_8m": 2_000_000}
# pseudo-particle selection: r_part, r_leaf from the paper's Table 1 runs; theta
# chosen so that the cloud yields about 1e5 pseudo-particles (102,908)
THETA = 0.065
L2_BYTES = 129 * 2 ** 20
# pseudo-particles (or particles) in the oracle's CPU sample of a workload
CPU_SAMPLE_TARGETS = 512


def parse():
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--workload", choices=tuple(WORKLOADS), default="pseudo_1e6",
                    help="pseudo_1e6: 1e6-particle cloud through the tree and pseudo-particles (the "
                         "benchmark); pseudo_2e5: the same path on 2e5 particles (profiling case); "
                         "sphere_1e5: 1e5 particles mapped directly (smaller case); "
                         "batched_64: 64 independent snapshots of 1e3-1e5 particles through map_batch; "
                         "full_8m: 8e6 particles and 2e6 cells (accuracy on a pair sample); "
                         "direct_8m: the same cloud with every particle mapped (tree off)")
    ap.add_argument("--workers", type=int, default=8, help="batched_64: host threads (streams) of map_batch")
    ap.add_argument("--precision", choices=("mixed", "fp64"), default="mixed")
    ap.add_argument("--theta", type=float, default=THETA)
    ap.add_argument("--fp64-threshold", type=float, default=1e-5)
    ap.add_argument("--err-ulps", type=int, default=0,
                    help="factor of the mixed pass's FP32 error estimate in units of 2^-24 (0: 8)")
    ap.add_argument("--h-tol", type=float, default=1e-13,
                    help="Newton tolerance |dh|/h_0 of the node h-solver; the paper runs 1e-2")
    ap.add_argument("--accuracy-pairs", type=int, default=-1,
                    help="pairs compared with the FP64 path in mixed mode: a random sample of this size, 0 for "
                         "all pairs (default: the workload's sample size, all pairs where none is set)")
    ap.add_argument("--split", choices=("replicas", "spatial"), default="replicas",
                    help="N > 1: an independent replica of the problem per rank (weak scaling), or one problem "
                         "split over the ranks by Morton ranges of its cells with one all-reduce of the "
                         "inverse mapping's sums (strong scaling)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="mixed mode: keep the FP32 pass's default launch shape instead of tuning it on the workload "
                         "(map_autotune, cached by device and workload in --cache/autotune.json)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cache", default=os.path.join(ROOT, "_cache"))
    return ap.parse_args()


def load_workload(args):
    from paper_2410_15227_gb300 import inputs
    if args.workload == "pseudo_1e6":
        w = inputs.cached(inputs.workload_pseudo_1e6, cache_dir=args.cache)
        w.params["theta"] = args.theta
    elif args.workload == "pseudo_2e5":
        w = inputs.cached(inputs.workload_pseudo_2e5, cache_dir=args.cache)
        if args.theta == THETA:   # the default theta is the 1e6 cloud's
            args.theta = w.params["theta"]
        w.params["theta"] = args.theta
    elif args.workload in ("full_8m", "direct_8m"):
        w = inputs.cached(inputs.workload_full_8m, cache_dir=args.cache)
        w.params["theta"] = args.theta
    else:
        w = inputs.cached(inputs.workload_sphere_100k, cache_dir=args.cache)
        w.params = dict(inputs.PSEUDO_PARAMS)
    return w


# ---------------------------------------------------------------------------
# clocks
# ---------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.file = None

    def start(self):
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.file,
                stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.file.flush()
        self.file.seek(0)
        rows = [r.strip().split(",") for r in self.file.read().strip().splitlines() if r.strip()]
        os.unlink(self.file.name)
        sm, mx, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for r in rows:
            try:
                sm.append(float(r[0]))
                mx.append(float(r[1]))
                for nm, v in zip(names, r[3:7]):
                    if "Active" in v and "Not" not in v:
                        reasons.add(nm)
            except (ValueError, IndexError):
                continue
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------

def run_ours(args, rank, world):
    import numpy as np
    import torch

    from paper_2410_15227_gb300 import api

    dev_index = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev_index)
    device = torch.device("cuda", dev_index)
    w = load_workload(args)
    ctx = api.Context(dev_index)
    dv = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=device)
    X = [dv(a) for a in (w.x, w.y, w.z, w.m, w.h)]
    f_np = np.random.default_rng([5, 3]).random(w.ngen)
    spatial = args.split == "spatial"
    if spatial:
        # one problem over the ranks: generators in Morton order, this rank's
        # contiguous range of cells
        from paper_2410_15227_gb300 import partition
        order = partition.morton_order(w.gx, w.gy, w.gz, w.box)
        G = [dv(a[order]) for a in (w.gx, w.gy, w.gz)]
        f_cell = dv(f_np[order])
        cell_range = partition.contiguous_ranges(w.ngen, world)[rank]
    else:
        G = [dv(a) for a in (w.gx, w.gy, w.gz)]
        f_cell = dv(f_np)
        cell_range = None
    src = np.zeros((1, 3))
    P = api.Params(r_part=w.params["r_part"], r_leaf=w.params["r_leaf"], theta=args.theta,
                   h_fact=w.params["h_fact"], h_tol=args.h_tol,
                   precision=1 if args.precision == "mixed" else 0,
                   fp64_threshold=args.fp64_threshold, fp32_err_ulps=err_ulps(args))
    stream = torch.cuda.current_stream(device)
    peaks = ctx.measure_peaks()
    map_ms = []
    kernel_ms = []   # (main pass, FP64 recompute) of each timed map_exact, from the library's events

    pseudo = WORKLOADS[args.workload][1]

    def step(x, y, z, m, h, gx, gy, gz, fc, record=False):
        if pseudo:
            tree = api.build_tree(ctx, x, y, z, m, w.box, 8)
            ps = api.make_pseudo_particles(ctx, tree, h, src, P)
            g = ps.get()
        else:
            tree = ps = None
            g = dict(x=x, y=y, z=z, h=h, m=m)
        if spatial:
            vor = api.build_voronoi_cells(ctx, gx, gy, gz, w.box, *cell_range, P)
            pr = api.find_pairs_cells(ctx, g["x"], g["y"], g["z"], g["h"], vor, *cell_range)
        else:
            vor = api.build_voronoi(ctx, gx, gy, gz, w.box, P)
            pr = api.find_pairs(ctx, g["x"], g["y"], g["z"], g["h"], vor)
        if record:
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
        wts, rho, wsum, nf = api.map_exact(ctx, pr, g["x"], g["y"], g["z"], g["h"], g["m"], vor, P,
                                           want_count=not record)
        if record:
            e1.record(stream)
            map_ms.append((e0, e1))
            kernel_ms.append(ctx.map_times())
        if spatial:
            # this rank's part of the inverse mapping's sums, added over the ranks
            from paper_2410_15227_gb300 import partition
            num = torch.zeros(g["x"].numel(), dtype=torch.float64, device=device)
            den = torch.zeros_like(num)
            api.map_back_sums(ctx, pr, wts, fc, num, den)
            partition.reduce_sums(num, den)
            if world > 1 and wsum is not None:   # each particle's weight sum, over every rank's cells
                torch.distributed.all_reduce(wsum)
            f = num / den
            fp = api.inherit(ctx, ps, tree, f) if pseudo else None
        else:
            f, fp = api.map_back(ctx, pr, wts, fc, ps, tree)
        return dict(npairs=pr.info()[0], npseudo=ps.info()[0] if pseudo else w.n, nfp64=nf, rho=rho, fp=fp, wsum=wsum,
                    w=wts, pr=pr, g=g, vor=vor)

    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=device)
    for _ in range(max(args.warmup, 0)):
        out = step(*X, *G, f_cell)
    torch.cuda.synchronize()
    tuned = None
    if args.precision == "mixed" and not args.no_autotune:
        # the FP32 pass's launch shape, tuned on this workload's pairs (each shape is
        # deterministic; the shapes agree to the mixed mode's tolerance)
        g = out["g"]
        tune = lambda: api.map_autotune(ctx, out["pr"], g["x"], g["y"], g["z"], g["h"], out["vor"], P)
        cache = os.path.join(args.cache, "autotune.json") if args.cache else None
        variant, ms, hit = api.autotune_cached(ctx, f"{args.workload}_theta{args.theta}", cache, tune)
        P.fp32_variant = variant
        tuned = {"variant": variant, "ms_per_variant": ms, "cached": hit}

    # accuracy of the mixed path against the FP64 path on the same pairs
    acc = {}
    nsample = args.accuracy_pairs if args.accuracy_pairs >= 0 else ACCURACY_SAMPLE.get(args.workload, 0)
    if args.precision == "mixed" and nsample > 0:
        acc = sampled_accuracy(api, ctx, out, nsample, device, [float(b) for b in w.box])
    elif args.precision == "mixed":
        P64 = api.Params(precision=0)
        g = out["g"]
        w64, rho64, u64, _ = api.map_exact(ctx, out["pr"], g["x"], g["y"], g["z"], g["h"], g["m"],
                                           out["vor"], P64)
        # relative errors where the 1e-5 relative target applies, i.e. above
        # the absolute floor 1e-14 / 1e-5; the absolute error over all pairs
        dw = (out["w"] - w64).abs()
        big = w64.abs() >= 1e-9
        rel = dw[big] / w64[big].abs()
        rrel = (out["rho"] - rho64).abs() / rho64.abs().clamp_min(1e-300)
        inner = u64 > 1 - 1e-12
        tot64 = (rho64 * 1.0).sum()
        acc = {"max_rel_err_w_vs_fp64": float(rel.max()), "rms_rel_err_w_vs_fp64": float(rel.pow(2).mean().sqrt()),
               "rel_err_over": "pairs with |w| >= 1e-9",
               "max_abs_err_w_vs_fp64": float(dw.max()),
               "pairs_over_1e-5_rel_plus_1e-14_abs": int((dw > 1e-5 * w64.abs() + 1e-14).sum()),
               "max_rel_err_rho_vs_fp64": float(rrel.max()),
               "max_abs_unity_err": float((out["wsum"][inner] - 1).abs().max()) if bool(inner.any()) else None,
               "fp64_recomputed_frac": out["nfp64"] / max(out["npairs"], 1)}
        del tot64
        # FP64 map_exact throughput on the same pairs (reported beside the mixed one)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        flush.zero_()
        e0.record(stream)
        api.map_exact(ctx, out["pr"], g["x"], g["y"], g["z"], g["h"], g["m"], out["vor"], P64)
        e1.record(stream)
        torch.cuda.synchronize()
        acc["fp64_map_exact_pairs_per_s"] = out["npairs"] / (e0.elapsed_time(e1) * 1e-3)
    del out

    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(dev_index)
    clocks.start()
    ctx.set_timing(True)
    launches0 = ctx.launches
    step_ms, npairs = [], 0
    for _ in range(args.steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        out = step(*X, *G, f_cell, record=True)
        e1.record(stream)
        npairs += out["npairs"]
        step_ms.append((e0, e1))
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    ck = clocks.stop()
    ctx.set_timing(False)
    launches = ctx.launches - launches0
    t_ms = sum(a.elapsed_time(b) for a, b in step_ms)
    t_map = [a.elapsed_time(b) for a, b in map_ms[-args.steps:]]
    tmax, units = reduce_over_ranks(t_ms, npairs, world, device)
    value = units / (tmax * 1e-3)
    res = dict(metric=METRIC, value=value, unit="pairs/s", n_gpus=world, steps=args.steps,
               warmup=args.warmup, ms_per_step=tmax / args.steps, higher_is_better=True,
               scaling="strong" if spatial else "weak", vs_baseline=None,
               dtype="f32+f64" if args.precision == "mixed" else "f64", data="synthetic",
               config={"workload": WORKLOADS[args.workload][0], "particles": w.n, "cells": w.ngen,
                       "pseudo_particles": out["npseudo"] if pseudo else None, "pairs_per_step": out["npairs"],
                       "theta": args.theta, "r_part": w.params["r_part"], "r_leaf": w.params["r_leaf"],
                       "precision": args.precision, "fp64_threshold": args.fp64_threshold, "h_tol": args.h_tol,
                       "fp32_err_ulps": err_ulps(args), "fp32_variant": P.fp32_variant,
                       "l2": "flushed between steps (258 MiB write)",
                       "parallelism": (f"spatial split x{world} (this rank's cells {cell_range[0]}..{cell_range[1]})"
                                       if spatial else f"replicas x{world}")},
               map_exact_ms=statistics.mean(t_map), map_exact_pairs_per_s=out["npairs"] / (statistics.mean(t_map) * 1e-3),
               accuracy=acc, gpu_launches=launches, clocks=ck, autotune=tuned)
    k_main = statistics.mean(k[0] for k in kernel_ms)
    k_re = statistics.mean(k[1] for k in kernel_ms)
    res["map_exact_kernels_ms"] = {"main": k_main, "fp64_recompute": k_re}
    res["roofline"] = roofline(out["npairs"], k_main, args.precision, args.workload, peaks,
                               ck["sm_mhz"] if ck else None)
    res["measured_peaks"] = peaks
    if not args.no_e2e:
        res["e2e"] = run_e2e(args, w, step, device)
    return res


def err_ulps(args):
    """Factor of the mixed pass's error estimate, 8 ulps unless given."""
    return args.err_ulps if args.err_ulps > 0 else 8


def run_batched(args, rank, world):
    """64 independent snapshots (N_s log-uniform in [1e3, 1e5], a quarter as
    many sites) through map_batch: the front stages per snapshot on host
    threads with a stream each, then one mapping of every pair of the batch.
    The FP32 pass's launch shape is tuned once on the batch (map_autotune,
    cached by device and workload in --cache/autotune.json).  The work spans
    several streams and map_batch returns when all have finished, so a step is
    timed by the host clock between two device synchronisations.  Beside it:
    the one-worker step, and the batch mapped in FP64 (the mapping's device
    time and the cell densities' difference)."""
    import numpy as np
    import torch

    from paper_2410_15227_gb300 import api, inputs

    dev_index = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev_index)
    device = torch.device("cuda", dev_index)
    ws = inputs.workload_batched()
    dv = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=device)
    snaps = [dict(x=dv(w.x), y=dv(w.y), z=dv(w.z), m=dv(w.m), h=dv(w.h), gx=dv(w.gx), gy=dv(w.gy), gz=dv(w.gz),
                  box=w.box, sources=np.zeros((1, 3)), f_cell=dv(np.random.default_rng([5, s]).random(w.ngen)))
             for s, w in enumerate(ws)]
    pp = inputs.PSEUDO_PARAMS
    P = api.Params(r_part=pp["r_part"], r_leaf=pp["r_leaf"], theta=args.theta, h_fact=pp["h_fact"],
                   h_tol=args.h_tol, precision=1 if args.precision == "mixed" else 0,
                   fp64_threshold=args.fp64_threshold, fp32_err_ulps=err_ulps(args))
    flush = torch.empty(2 * L2_BYTES // 8, dtype=torch.float64, device=device)
    ctx = api.Context(dev_index)
    peaks = ctx.measure_peaks()

    def step(nworkers, params, tune=False):
        flush.zero_()
        torch.cuda.synchronize()
        info = {}
        t = time.perf_counter()
        res, launches = api.map_batch(dev_index, snaps, params, nworkers=nworkers, tune=tune, info=info)
        torch.cuda.synchronize()
        return (time.perf_counter() - t) * 1e3, sum(r["npairs"] for r in res), launches, res, info

    tuned = None
    if args.precision == "mixed":
        def tune():
            _, _, _, _, info = step(args.workers, P, tune=True)
            return info["variant"], None
        cache = os.path.join(args.cache, "autotune.json") if args.cache else None
        variant, _, hit = api.autotune_cached(ctx, f"batched_64_theta{args.theta}", cache, tune)
        P.fp32_variant = variant
        tuned = {"variant": variant, "cached": hit}
    for _ in range(args.warmup):
        out = step(args.workers, P)
    serial_ms = min(step(1, P)[0] for _ in range(2))
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(dev_index)
    clocks.start()
    t_ms, npairs, launches, map_ms = 0.0, 0, 0, []
    for _ in range(args.steps):
        ms, n, nl, res, info = step(args.workers, P)
        t_ms += ms
        npairs += n
        launches += nl
        map_ms.append(info["map_ms"])
    if world > 1:
        torch.distributed.barrier()
    ck = clocks.stop()
    tmax, units = reduce_over_ranks(t_ms, npairs, world, device)
    per_step = npairs // args.steps
    k_main = statistics.mean(m[0] for m in map_ms)
    k_re = statistics.mean(m[1] for m in map_ms)
    out = dict(metric=METRIC, value=units / (tmax * 1e-3), unit="pairs/s", n_gpus=world, steps=args.steps,
               warmup=args.warmup, ms_per_step=tmax / args.steps, higher_is_better=True, scaling="weak",
               vs_baseline=None, dtype="f32+f64" if args.precision == "mixed" else "f64", data="synthetic",
               config={"workload": WORKLOADS[args.workload][0], "snapshots": len(ws),
                       "particles": int(sum(w.n for w in ws)), "cells": int(sum(w.ngen for w in ws)),
                       "pseudo_particles": int(sum(r["npseudo"] for r in res)), "pairs_per_step": per_step,
                       "theta": args.theta, "r_part": pp["r_part"], "r_leaf": pp["r_leaf"],
                       "precision": args.precision, "fp64_threshold": args.fp64_threshold, "h_tol": args.h_tol,
                       "workers": args.workers, "fp32_variant": P.fp32_variant,
                       "timing": "host clock between device syncs around map_batch",
                       "l2": "flushed between steps (258 MiB write)", "parallelism": f"replicas x{world}"},
               map_exact_kernels_ms={"main": k_main, "fp64_recompute": k_re},
               map_exact_pairs_per_s=per_step / ((k_main + k_re) * 1e-3), autotune=tuned,
               serial_ms_per_step=serial_ms, serial_pairs_per_s=per_step / (serial_ms * 1e-3),
               gpu_launches=launches, clocks=ck, measured_peaks=peaks, e2e=None, cpu_baseline=None)
    out["roofline"] = roofline(per_step, k_main, args.precision, "pseudo_1e6", peaks, ck["sm_mhz"] if ck else None)
    if out["roofline"]:
        out["roofline"]["work"] += " (the 1e6 cloud's count, same profile)"
    if args.precision == "mixed":
        # the same batch with every pair in FP64: the mapping's time, and how far
        # the mixed cell densities are from the FP64 ones
        P64 = api.Params(r_part=pp["r_part"], r_leaf=pp["r_leaf"], theta=args.theta, h_fact=pp["h_fact"],
                         h_tol=args.h_tol, precision=0)
        _, _, _, res64, info64 = step(args.workers, P64)
        rel = max(float(((a["rho"] - b["rho"]).abs() / b["rho"].abs().clamp_min(1e-300)).max())
                  for a, b in zip(res, res64))
        out["fp64"] = {"map_exact_ms": info64["map_ms"][0],
                       "map_exact_pairs_per_s": per_step / (info64["map_ms"][0] * 1e-3),
                       "max_rel_err_rho_mixed_vs_fp64": rel,
                       "fp64_recomputed_frac_mixed": sum(r["nfp64"] for r in res) / max(per_step, 1)}
    return out


def sampled_accuracy(api, ctx, out, nsample, device, box, seed=11):
    """Mixed against FP64 weights on a random sample of the pairs (a subset
    of the (j, i)-sorted list stays sorted), and the partition of unity
    sum_j w_ij = 1 over the pseudo-particles whose kernel lies inside the
    box, for which it holds exactly."""
    import torch
    pr, g, vor = out["pr"], out["g"], out["vor"]
    npairs, npseudo, _ = pr.info()
    pp = pr.get()
    gen = torch.Generator(device=device)
    gen.manual_seed(seed)
    k = min(nsample, npairs)
    idx = torch.randperm(npairs, device=device, generator=gen)[:k].sort().values
    sub = api.pairs_from_list(ctx, pp["pair_i"][idx].contiguous(), pp["pair_j"][idx].contiguous(), npseudo, vor)
    del pp
    w64, _, _, _ = api.map_exact(ctx, sub, g["x"], g["y"], g["z"], g["h"], g["m"], vor, api.Params(precision=0),
                                 want_wsum=False)
    wm = out["w"][idx]
    inside = ((g["x"] - box[0]).minimum(box[1] - g["x"]).minimum(g["y"] - box[2]).minimum(box[3] - g["y"])
              .minimum(g["z"] - box[4]).minimum(box[5] - g["z"])) >= 2 * g["h"]
    dw = (wm - w64).abs()
    big = w64.abs() >= 1e-9
    rel = dw[big] / w64[big].abs()
    over = dw > 1e-5 * w64.abs() + 1e-14
    return {"max_rel_err_w_vs_fp64": float(rel.max()), "rms_rel_err_w_vs_fp64": float(rel.pow(2).mean().sqrt()),
            "rel_err_over": "pairs with |w| >= 1e-9", "max_abs_err_w_vs_fp64": float(dw.max()),
            "pairs_over_1e-5_rel_plus_1e-14_abs": int(over.sum()), "sampled_pairs": int(k),
            "max_abs_unity_err": float((out["wsum"][inside] - 1).abs().max()),
            "unity_over": "pseudo-particles whose 2h sphere lies inside the box",
            "fp64_recomputed_frac": out["nfp64"] / max(npairs, 1)}


def reduce_over_ranks(t_ms, units, world, device):
    """Whole-job figures across ranks: the slowest rank's timed milliseconds
    and the units (pairs) all ranks processed.  One process per GPU; on one
    rank this is the identity."""
    if world == 1:
        return float(t_ms), float(units)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(t_ms)], dtype=torch.float64, device=device)
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


# Algorithmic work of map_exact per pair (the method's work, section 8(d)):
# the oracle's closed form, counted operation by operation by its counting
# build on the complete pair lists of 64 random (pseudo-)particles of each
# workload (`python -m oracle.count_work`): right sub-triangles evaluated,
# FP64 additions/subtractions + multiplications + divisions, square roots and
# transcendental calls (atan2, asinh, pow) per pair.
ALGO_WORK = {
    "pseudo_1e6": dict(subtriangles=163.76, flops=41824.8, sqrt=1021.39, transcendental=2286.21, pairs=14042),
    "pseudo_2e5": dict(subtriangles=162.86, flops=41708.6, sqrt=1017.31, transcendental=2280.04, pairs=13422),
    "sphere_1e5": dict(subtriangles=163.63, flops=46702.9, sqrt=1064.1, transcendental=2529.7, pairs=2734),
}
# Implementation work of the FP32 pass per pair (what the kernel executes,
# float-float bookkeeping included), for the utilisation figure beside the
# algorithmic one: the cell's faces, the faces within reach (D < 2 and R < 2 in
# units of h) and their edges, counted over random pairs of each workload with
# a CPU model of the FP32 pass (6,000 pairs of the 1e6 cloud, 3,683 of the 1e5
# sphere), and the quadrature's 4-node slots (a 4-point segment, or half of an
# 8-point sub-piece), counted over every pair of one launch by an instrumented
# build.
WORK = {
    "pseudo_1e6": dict(faces=15.64, faces_used=11.33, edges_used=60.65, slots=88.43),
    "sphere_1e5": dict(faces=15.23, faces_used=7.93, edges_used=43.36, slots=72.05),
}
# Work of the FP32 pass per unit, counted in its source (FMA = 2 flops):
#  - per quadrature node 53 FP32 flops (the node's place relative to its
#    segment's start, sinh, cosh and tau - ts from expm1, Q from rsqrt and a
#    Newton step, Q^2 - R^2 from the offset: 33; the kernel piece's integrand
#    about 20) and 5 SFU operations (expm1, the reciprocals of 1 + expm1,
#    Q + R and cosh, and rsqrt for Q);
#  - per edge of a face within reach 185 FP32 flops of float-float geometry
#    (two offset dot products, four products, four sums) and segment set-up
#    (lengths in s from the offsets, the differences at the start);
#  - per face 60 (float-float plane distance and, for faces within reach,
#    the face constants), and 18 per edge of a face within reach for the FP32
#    distance to the polygon;
#  - per 4-node slot 14 for the float-float accumulation and 6 for the
#    segment start's sinh and cosh (ts / A, and sqrt(1 + (ts/A)^2) by rsqrt
#    and a Newton step), formed where the slot is evaluated;
#  - per pair about 30 FP64 flops (r = x - g, 1/h, the final sums).
FP32_FLOPS_NODE, SFU_OPS_NODE = 53, 5
FP32_FLOPS_EDGE, FP32_FLOPS_FACE, FP32_FLOPS_POLY_EDGE, FP32_FLOPS_SLOT = 185, 60, 18, 20
FP64_FLOPS_PAIR = 30
# DRAM traffic of one k_map_fp32 launch per pair (ncu, dram__bytes_read.sum +
# dram__bytes_write.sum over the pairs of the launch), per workload, from a
# capture of the current kernel (profiles/k_map_fp32_dram_pseudo_1e6.md)
TRAFFIC_PER_PAIR = {"pseudo_1e6": 108.94}


def nominal_peaks(sm_count, mhz):
    """Nominal rates from the unit counts at a clock: FP32 128 lanes x 2 flops,
    FP64 2 FMA x 2 flops, SFU 16 operations per SM per clock."""
    f = sm_count * mhz * 1e6
    return dict(fp32_tflops=f * 128 * 2 / 1e12, fp64_tflops=f * 2 * 2 / 1e12, xu_tops=f * 16 / 1e12)


def roofline(npairs, ms, precision, workload, peaks, clock_mhz=None):
    """Dominant kernel of map_exact: k_map_fp32 (mixed) or k_map_fp64 (FP64),
    both bound by arithmetic, not memory.  achieved = the method's algorithmic
    work (ALGO_WORK: the oracle-counted operations of the closed form per pair)
    x the launch's pairs / its CUDA-event time, against the measured peak of
    the pipe that executes it (em_measure_peaks: FP32 for the mixed pass, FP64
    for the FP64 path); the special-function rate (square roots and
    transcendental calls) against the measured SFU peak beside it, and the
    FP32 pass's own instruction-mix flops (WORK) as a utilisation figure."""
    aw = ALGO_WORK.get(workload)
    if aw is None or ms <= 0:   # per-pair work not counted for this workload
        return None
    t = ms * 1e-3
    nom = nominal_peaks(peaks["sm_count"], clock_mhz or peaks["sm_clock_mhz"])
    achieved = npairs * aw["flops"] / t / 1e12
    xu = npairs * (aw["sqrt"] + aw["transcendental"]) / t / 1e12
    pipe = "fp32" if precision == "mixed" else "fp64"
    peak = peaks["fp32_tflops"] if pipe == "fp32" else peaks["fp64_tflops"]
    tr = TRAFFIC_PER_PAIR.get(workload) if precision == "mixed" else None
    out = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
           "traffic": tr * npairs if tr else None,
           "kernel": "k_map_fp32" if pipe == "fp32" else "k_map_fp64", "pipe": pipe, "kernel_ms": ms,
           "work": f"{aw['flops']:.0f} FP64 operations of the closed form per pair (oracle-counted, "
                   f"{aw['subtriangles']:.1f} right sub-triangles)",
           "peak_source": f"measured ({pipe.upper()} FMA chains, em_measure_peaks)",
           "nominal_peak": nom[pipe + "_tflops"], "nominal_clock_mhz": clock_mhz or peaks["sm_clock_mhz"],
           "sfu": {"achieved": xu, "peak": peaks["xu_tops"], "unit": "Top/s", "frac": xu / peaks["xu_tops"],
                   "ops_per_pair": aw["sqrt"] + aw["transcendental"],
                   "work": "square roots and transcendental calls of the closed form per pair"}}
    wk = WORK.get(workload)
    if precision == "mixed" and wk is not None:
        nodes = 4 * wk["slots"]
        f32 = (FP32_FLOPS_NODE * nodes + FP32_FLOPS_SLOT * wk["slots"]
               + (FP32_FLOPS_EDGE + FP32_FLOPS_POLY_EDGE) * wk["edges_used"] + FP32_FLOPS_FACE * wk["faces"])
        impl = npairs * f32 / t / 1e12
        out["implementation"] = {"achieved": impl, "unit": "TFLOP/s", "frac": impl / peaks["fp32_tflops"],
                                 "flops_per_pair": f32,
                                 "work": "the FP32 pass's own flops per pair (float-float bookkeeping included)"}
    return out


def run_e2e(args, w, step, device):
    """Same metric through the public API with host buffers: pinned host -> device
    copies of the step's inputs and device -> host copies of its results are
    inside the timed region."""
    import numpy as np
    import torch
    host = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
            for a in (w.x, w.y, w.z, w.m, w.h, w.gx, w.gy, w.gz,
                      np.random.default_rng([5, 3]).random(w.ngen))]
    bi = sum(t.numel() * t.element_size() for t in host)
    stream = torch.cuda.current_stream(device)
    reps = max(1, min(args.steps, 3))
    # the results land in pinned host buffers, allocated once like the inputs;
    # the copies run on the library's stream (torch's current one), after the
    # step's kernels, and all of them finish inside the timed region
    res_h = {"rho": torch.empty(w.ngen, dtype=torch.float64, pin_memory=True),
             "fp": torch.empty(w.n, dtype=torch.float64, pin_memory=True)}
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    npairs, bo = 0, 0
    for _ in range(reps):
        dev_in = [t.to(device, non_blocking=True) for t in host]
        out = step(*dev_in)
        bo = 0
        for key in ("rho", "fp"):
            d = out[key]
            if d is None:
                continue
            if key not in res_h or res_h[key].shape != d.shape:
                res_h[key] = torch.empty(d.shape, dtype=d.dtype, pin_memory=True)
            res_h[key].copy_(d, non_blocking=True)
            bo += d.numel() * d.element_size()
        npairs += out["npairs"]
    stream.synchronize()
    dt = time.perf_counter() - t0
    return {"value": npairs / dt, "unit": "pairs/s", "h2d_bytes_per_step": bi, "d2h_bytes_per_step": bo,
            "steps": reps}


# ---------------------------------------------------------------------------
# CPU oracle (baseline and reference arm)
# ---------------------------------------------------------------------------

def oracle_sample(w, theta, ntarget=CPU_SAMPLE_TARGETS, seed=7, pseudo=True):
    """A bounded sample of the same workload, built by the FP64 CPU oracle
    alone (oracle.workload_sample): `ntarget` random pseudo-particles (or
    particles, for a workload mapped directly) with the cells of the
    generators within their 2h and the pairs among these."""
    import oracle
    return oracle.workload_sample(w, theta, ntarget=ntarget, seed=seed, pseudo=pseudo)


def time_oracle(parts, cells, pairs, reps=1, nthreads=None):
    import oracle
    nt = nthreads or oracle.nthreads_default()
    t0 = time.perf_counter()
    for _ in range(reps):
        oracle.map_exact(pairs, *parts, cells, nthreads=nt)
    dt = time.perf_counter() - t0
    return pairs.n * reps / dt, nt, dt


def _sample_text(pairs, cells, nt, ntarget, pseudo=True):
    who = (f"{ntarget} random pseudo-particles (oracle tree, selection and h-solver on the cloud)"
           if pseudo else f"{ntarget} random particles of the cloud")
    return (f"oracle map_exact (FP64, OpenMP, {nt} threads) on {pairs.n} distinct pairs of {who} with the "
            f"oracle's brute-force cells of the {cells.ncell} generators within their 2h; every pass maps all "
            f"of them")


def cpu_baseline(args, w):
    """The oracle on a bounded sample of the workload: one cold pass over its
    distinct pairs, then whole passes for about 10 s on all host cores, one
    pass on one core; and the sample's algorithmic work per pair, counted by
    the oracle's counting build."""
    import oracle
    pseudo = WORKLOADS[args.workload][1]
    parts, cells, pairs = oracle_sample(w, args.theta, pseudo=pseudo)
    v0, nt, dt = time_oracle(parts, cells, pairs, 1)
    reps = max(1, int(10.0 / max(dt, 1e-3)))
    v, nt, dt = time_oracle(parts, cells, pairs, reps)
    v1, _, _ = time_oracle(parts, cells, pairs, 1, nthreads=1)
    _, counts = oracle.count_map_exact(pairs, *parts, cells)
    work = {k: float(c) for k, c in zip(oracle.WORK_FIELDS, counts.mean(axis=0))}
    return {"value": v, "unit": "pairs/s", "cores": nt, "kind": "oracle",
            "sample": _sample_text(pairs, cells, nt, CPU_SAMPLE_TARGETS, pseudo) + f"; {reps} passes in {dt:.1f} s",
            "first_pass_value": v0, "single_core_value": v1, "distinct_pairs": pairs.n,
            "oracle_work_per_pair": work}


def run_reference(args, rank, world):
    if rank != 0:
        return None
    if args.workload == "batched_64":
        return {"impl": "reference", "unavailable": "the oracle arm times samples of one snapshot; "
                                                    "batched_64 is measured against map_batch with one worker"}
    w = load_workload(args)
    pseudo = WORKLOADS[args.workload][1]
    parts, cells, pairs = oracle_sample(w, args.theta, pseudo=pseudo)
    _, _, dt = time_oracle(parts, cells, pairs, 1)
    reps = max(1, int(2.0 / max(dt, 1e-3)))    # about 2 s of oracle work per step
    for _ in range(max(args.warmup, 0)):
        time_oracle(parts, cells, pairs, reps)
    t0 = time.perf_counter()
    n = 0
    for _ in range(args.steps):
        v, nt, dt = time_oracle(parts, cells, pairs, reps)
        n += pairs.n * reps
    t = time.perf_counter() - t0
    value = n / t
    sample = _sample_text(pairs, cells, nt, CPU_SAMPLE_TARGETS, pseudo) + f"; {reps} passes per step"
    return dict(metric=METRIC, value=value, unit="pairs/s", n_gpus=world, steps=args.steps,
                warmup=args.warmup, ms_per_step=t / args.steps * 1e3, higher_is_better=True,
                scaling="weak", vs_baseline=None, dtype="f64", data="synthetic",
                config={"workload": WORKLOADS[args.workload][0], "particles": w.n, "cells": w.ngen,
                        "sampled_cells": cells.ncell,
                        "pairs_per_step": pairs.n * reps, "theta": args.theta},
                impl="reference",
                cpu_baseline={"value": value, "unit": "pairs/s", "cores": nt, "kind": "oracle", "sample": sample},
                e2e={"value": value, "unit": "pairs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
                gpu_launches=0)


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        res = run_reference(args, rank, world)
        if res is not None:
            print(json.dumps(res))
        return
    if world > 1:
        import torch
        torch.distributed.init_process_group("nccl")
    if args.workload == "batched_64":
        res = run_batched(args, rank, world)
        if rank == 0:
            print(json.dumps(res))
        if world > 1:
            import torch
            torch.distributed.destroy_process_group()
        return
    res = run_ours(args, rank, world)
    if rank == 0:
        if not args.no_cpu_baseline:
            res["cpu_baseline"] = cpu_baseline(args, load_workload(args))
        print(json.dumps(res))
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
