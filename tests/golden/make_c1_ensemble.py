"""Writes tests/golden/c1_ensemble_1000.json: the FP64 CPU oracle's moments of the
32x32x64-cell workload (1e4 macroparticles at weight 100, 3 kV, dt 0.5 fs) over
1000 steps for 16 seeds, at steps 250, 500, 750 and 1000, per seed (so a test can
form ensemble means and their standard errors). It calls only the oracle and
the seeded workload generator.

    python tests/golden/make_c1_ensemble.py [--seeds 16] [--steps 1000] [--procs 8]
"""
from __future__ import annotations

import argparse
import json
import multiprocessing as mp
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
OUT = os.path.join(ROOT, "tests", "golden", "c1_ensemble_1000.json")
CHECKPOINTS = (250, 500, 750, 1000)
KEYS = ("count", "kinetic", "n_ionization", "n_elastic", "abs_anode", "abs_cathode", "field_energy", "injected")


def one_run(args):
    seed, steps = args
    sys.path.insert(0, ROOT)
    import oracle
    from paper_2606_05893_gb300 import workloads as W
    wl = W.config_small(seed=seed)
    o = oracle.Oracle(wl)
    t0 = time.perf_counter()
    rows = {}
    done = 0
    for cp in CHECKPOINTS:
        if cp > steps:
            break
        o.step(cp - done)
        done = cp
        m = o.moments()
        rows[str(cp)] = {k: m[k] for k in KEYS}
    o.close()
    return seed, rows, time.perf_counter() - t0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--seeds", type=int, default=16)
    ap.add_argument("--first-seed", type=int, default=42)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--procs", type=int, default=8)
    a = ap.parse_args()
    sys.path.insert(0, ROOT)
    import oracle
    oracle.build()
    seeds = list(range(a.first_seed, a.first_seed + a.seeds))
    ctx = mp.get_context("spawn")
    with ctx.Pool(a.procs) as pool:
        res = pool.map(one_run, [(s, a.steps) for s in seeds])
    out = {"workload": "32x32x64 cells h=5nm, 1e4 macroparticles at weight 100, 3 kV, dt 0.5 fs (config_small)",
           "oracle": "FP64 CPU oracle, cg_rtol of the workload", "checkpoints": [c for c in CHECKPOINTS if c <= a.steps],
           "seeds": seeds, "runs": {str(s): rows for s, rows, _ in res},
           "seconds_per_run": {str(s): round(t, 1) for s, _, t in res}}
    with open(OUT, "w") as f:
        json.dump(out, f, indent=1)
    print("wrote", OUT, "in", round(max(t for _, _, t in res), 1), "s per run")


if __name__ == "__main__":
    main()
