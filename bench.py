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
    "sphere_1e5": ("sphere_100k_particles_25k_cells", False),
}
# pseudo-particle selection: r_part, r_leaf from the paper's Table 1 runs; theta
# chosen so that the cloud yields about 1e5 pseudo-particles (102,908)
THETA = 0.065
L2_BYTES = 129 * 2 ** 20


def parse():
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--workload", choices=tuple(WORKLOADS), default="pseudo_1e6",
                    help="pseudo_1e6: 1e6-particle cloud through the tree and pseudo-particles (the "
                         "benchmark); sphere_1e5: 1e5 particles mapped directly (smaller case)")
    ap.add_argument("--precision", choices=("mixed", "fp64"), default="mixed")
    ap.add_argument("--theta", type=float, default=THETA)
    ap.add_argument("--fp64-threshold", type=float, default=1e-5)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cache", default=os.path.join(ROOT, "_cache"))
    return ap.parse_args()


def load_workload(args):
    from paper_2410_15227_gb300 import inputs
    if args.workload == "pseudo_1e6":
        w = inputs.cached(inputs.workload_pseudo_1e6, cache_dir=args.cache)
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
    G = [dv(a) for a in (w.gx, w.gy, w.gz)]
    f_cell = dv(np.random.default_rng([5, 3]).random(w.ngen))
    src = np.zeros((1, 3))
    P = api.Params(r_part=w.params["r_part"], r_leaf=w.params["r_leaf"], theta=args.theta,
                   h_fact=w.params["h_fact"], h_tol=1e-13,
                   precision=1 if args.precision == "mixed" else 0,
                   fp64_threshold=args.fp64_threshold)
    stream = torch.cuda.current_stream(device)
    map_ms = []

    pseudo = WORKLOADS[args.workload][1]

    def step(x, y, z, m, h, gx, gy, gz, fc, record=False):
        if pseudo:
            tree = api.build_tree(ctx, x, y, z, m, w.box, 8)
            ps = api.make_pseudo_particles(ctx, tree, h, src, P)
            g = ps.get()
        else:
            tree = ps = None
            g = dict(x=x, y=y, z=z, h=h, m=m)
        vor = api.build_voronoi(ctx, gx, gy, gz, w.box, P)
        pr = api.find_pairs(ctx, g["x"], g["y"], g["z"], g["h"], vor)
        if record:
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
        wts, rho, wsum, nf = api.map_exact(ctx, pr, g["x"], g["y"], g["z"], g["h"], g["m"], vor, P)
        if record:
            e1.record(stream)
            map_ms.append((e0, e1))
        f, fp = api.map_back(ctx, pr, wts, fc, ps, tree)
        return dict(npairs=pr.info()[0], npseudo=ps.info()[0] if pseudo else w.n, nfp64=nf, rho=rho, fp=fp, wsum=wsum,
                    w=wts, pr=pr, g=g, vor=vor)

    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=device)
    for _ in range(max(args.warmup, 0)):
        out = step(*X, *G, f_cell)
    torch.cuda.synchronize()

    # accuracy of the mixed path against the FP64 path on the same pairs
    acc = {}
    if args.precision == "mixed":
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
    launches = ctx.launches - launches0
    t_ms = sum(a.elapsed_time(b) for a, b in step_ms)
    t_map = [a.elapsed_time(b) for a, b in map_ms[-args.steps:]]
    tmax = t_ms
    if world > 1:
        tt = torch.tensor([t_ms], device=device)
        torch.distributed.all_reduce(tt, op=torch.distributed.ReduceOp.MAX)
        tmax = float(tt.item())
    value = npairs * world / (tmax * 1e-3)
    res = dict(metric=METRIC, value=value, unit="pairs/s", n_gpus=world, steps=args.steps,
               warmup=args.warmup, ms_per_step=tmax / args.steps, higher_is_better=True,
               scaling="weak", vs_baseline=None,
               dtype="f32+f64" if args.precision == "mixed" else "f64", data="synthetic",
               config={"workload": WORKLOADS[args.workload][0], "particles": w.n, "cells": w.ngen,
                       "pseudo_particles": out["npseudo"] if pseudo else None, "pairs_per_step": out["npairs"],
                       "theta": args.theta, "r_part": w.params["r_part"], "r_leaf": w.params["r_leaf"],
                       "precision": args.precision, "fp64_threshold": args.fp64_threshold,
                       "l2": "flushed between steps (258 MiB write)", "parallelism": f"replicas x{world}"},
               map_exact_ms=statistics.mean(t_map), map_exact_pairs_per_s=out["npairs"] / (statistics.mean(t_map) * 1e-3),
               accuracy=acc, gpu_launches=launches, clocks=ck)
    res["roofline"] = roofline(out["npairs"], statistics.mean(t_map), args.precision)
    if not args.no_e2e:
        res["e2e"] = run_e2e(args, w, step, device)
    return res


def roofline(npairs, ms, precision):
    """Dominant kernel: the per-pair analytic integral (FP32 bulk pass in mixed
    mode), bound by the FP32 pipe.  Algorithmic work per pair: FLOPS_PER_PAIR
    (see the design doc); peak: 152 SMs x 128 FP32 lanes x 2 flop x 2.07 GHz."""
    flops_per_pair = FLOPS_PER_PAIR_F32 if precision == "mixed" else FLOPS_PER_PAIR_F64
    peak = 152 * 128 * 2 * 2.07e9 / 1e12 if precision == "mixed" else FP64_PEAK_TFLOPS
    achieved = npairs * flops_per_pair / (ms * 1e-3) / 1e12
    return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak, "traffic": None,
            "kernel": "k_map_fp32" if precision == "mixed" else "k_map_fp64",
            "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 x 2.07 GHz"}


# FP32 operations per pair of the bulk pass and FP64 per pair of the FP64 pass,
# counted on the 1e6-particle workload (measurement section)
FLOPS_PER_PAIR_F32 = 1.0e4
FLOPS_PER_PAIR_F64 = 1.0e4
FP64_PEAK_TFLOPS = 1.25


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
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    npairs, bo = 0, 0
    for _ in range(reps):
        dev_in = [t.to(device, non_blocking=True) for t in host]
        out = step(*dev_in)
        rho_h = out["rho"].to("cpu", non_blocking=False)
        fp_h = out["fp"].to("cpu", non_blocking=False)
        bo = rho_h.numel() * 8 + fp_h.numel() * 8
        npairs += out["npairs"]
    stream.synchronize()
    dt = time.perf_counter() - t0
    return {"value": npairs / dt, "unit": "pairs/s", "h2d_bytes_per_step": bi, "d2h_bytes_per_step": bo,
            "steps": reps}


# ---------------------------------------------------------------------------
# CPU oracle (baseline and reference arm)
# ---------------------------------------------------------------------------

def oracle_sample(w, theta, ntarget=64, seed=7, pseudo=True):
    """A bounded sample of the same workload, built by the FP64 CPU oracle
    alone: `ntarget` random pseudo-particles from its own tree and selection
    on the cloud (nodes get h from the oracle's h-solver against the whole
    population) -- or random particles when the workload maps particles
    directly -- the oracle's brute-force cells of every generator within 2h of
    them, and the oracle's pairs among these."""
    import numpy as np

    import oracle
    pr = w.params
    rng = np.random.default_rng(seed)
    if not pseudo:      # the particles themselves
        tg = np.sort(rng.choice(w.n, ntarget, replace=False))
        px, py, pz, h = w.x[tg], w.y[tg], w.z[tg], w.h[tg]
        return _sample_cells(w, px, py, pz, h)
    ps, tree, sel = oracle.make_pseudo_particles(w.x, w.y, w.z, w.m, w.h, w.box, np.zeros((1, 3)),
                                                 pr["r_part"], pr["r_leaf"], theta, h_fact=pr["h_fact"],
                                                 solve=False)
    tg = np.sort(rng.choice(ps.n, ntarget, replace=False))
    h = ps.h[tg].copy()
    node = ps.origin[tg] > 0
    if node.any():
        ids = sel.ref[tg[node]]
        h0 = oracle.h_initial(tree, ids, w.h, pr["h_fact"])
        h[node] = oracle.h_solve(tree.com[sel.pop_node], tree.com[ids], h0, pr["h_fact"], 1e-13, 50)[0]
    return _sample_cells(w, ps.x[tg], ps.y[tg], ps.z[tg], h)


def _sample_cells(w, px, py, pz, h):
    import numpy as np

    import oracle
    ntarget = px.shape[0]
    gen = np.stack([w.gx, w.gy, w.gz], 1)
    near = np.zeros(w.ngen, bool)
    for a in range(ntarget):
        near |= np.einsum("ij,ij->i", gen - (px[a], py[a], pz[a]), gen - (px[a], py[a], pz[a])) < 4 * h[a] ** 2
    cells = oracle.voronoi(w.gx, w.gy, w.gz, w.box, cells=np.flatnonzero(near))
    pairs = oracle.find_pairs(px, py, pz, h, cells)
    return (px, py, pz, h), cells, pairs


def time_oracle(parts, cells, pairs, reps=1):
    import oracle
    nt = oracle.nthreads_default()
    t0 = time.perf_counter()
    for _ in range(reps):
        oracle.map_exact(pairs, *parts, cells, nthreads=nt)
    dt = time.perf_counter() - t0
    return pairs.n * reps / dt, nt, dt


def _sample_text(pairs, cells, nt, pseudo=True):
    who = ("64 random pseudo-particles (oracle tree, selection and h-solver on the 1e6-particle cloud)"
           if pseudo else "64 random particles of the cloud")
    return (f"oracle map_exact (FP64, OpenMP, {nt} threads) on {pairs.n} pairs of {who} with the oracle's "
            f"brute-force cells of the {cells.ncell} generators within their 2h")


def cpu_baseline(args, w):
    pseudo = WORKLOADS[args.workload][1]
    parts, cells, pairs = oracle_sample(w, args.theta, pseudo=pseudo)
    v, nt, dt = time_oracle(parts, cells, pairs, 1)
    reps = max(1, int(15.0 / max(dt, 1e-3)))
    v, nt, dt = time_oracle(parts, cells, pairs, reps)
    return {"value": v, "unit": "pairs/s", "cores": nt, "kind": "oracle",
            "sample": _sample_text(pairs, cells, nt, pseudo) + f", x{reps} in {dt:.1f} s"}


def run_reference(args, rank, world):
    if rank != 0:
        return None
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
    sample = _sample_text(pairs, cells, nt, pseudo) + f", x{reps} per step"
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
