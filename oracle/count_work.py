"""Algorithmic work per mapped pair of the benchmark workloads, counted by the
oracle's counting build (count.cpp) on the complete pair lists of a random
sample of each workload's (pseudo-)particles, built by the oracle alone
(workload_sample with complete=True).  Test infrastructure: prints the mean
counts per pair -- right sub-triangles, FP64 additions, multiplications,
divisions, square roots and transcendental calls of the closed form -- which
the benchmark's roofline takes as the method's work per pair.

    python -m oracle.count_work [--targets 64] [--workloads pseudo_1e6 pseudo_2e5 sphere_1e5]
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from paper_2410_15227_gb300 import inputs  # noqa: E402

WORKLOADS = {
    "pseudo_1e6": (inputs.workload_pseudo_1e6, True),
    "pseudo_2e5": (inputs.workload_pseudo_2e5, True),
    "sphere_1e5": (inputs.workload_sphere_100k, False),
}


def main():
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--targets", type=int, default=64)
    ap.add_argument("--seed", type=int, default=9)
    ap.add_argument("--workloads", nargs="+", default=list(WORKLOADS))
    ap.add_argument("--cache", default=os.path.join(ROOT, "_cache"))
    args = ap.parse_args()
    out = {}
    for name in args.workloads:
        make, pseudo = WORKLOADS[name]
        w = inputs.cached(make, cache_dir=args.cache)
        if not getattr(w, "params", None):
            w.params = dict(inputs.PSEUDO_PARAMS)
        theta = w.params.get("theta", inputs.THETA_1E6)
        t0 = time.perf_counter()
        parts, cells, pairs = oracle.workload_sample(w, theta, ntarget=args.targets, seed=args.seed,
                                                     pseudo=pseudo, complete=True)
        _, counts = oracle.count_map_exact(pairs, *parts, cells)
        mean = counts.astype(np.float64).mean(axis=0)
        row = {k: round(float(v), 2) for k, v in zip(oracle.WORK_FIELDS, mean)}
        row["fp64_ops"] = round(float(mean[1] + mean[2] + mean[3]), 1)
        row["pairs"] = int(pairs.n)
        row["targets"] = args.targets
        row["seconds"] = round(time.perf_counter() - t0, 1)
        out[name] = row
        print(json.dumps({name: row}), flush=True)


if __name__ == "__main__":
    main()
