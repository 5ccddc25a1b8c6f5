"""1000 steps of the 32x32x64-cell workload (1e4 macroparticles at weight 100,
3 kV, dt 0.5 fs) on the GPU, FP64 and mixed stores, against the FP64 CPU
oracle's ensemble over the same 16 seeds (tests/golden/c1_ensemble_1000.json,
written by tests/golden/make_c1_ensemble.py, which calls only the oracle).

The runs are chaotic (a last-bit difference of a deposit sum moves a particle
across a cell or a collision threshold within tens of steps), so individual
runs are compared as samples of one ensemble: at steps 250, 500, 750 and 1000
the ensemble means of the particle counts and kinetic energies per species, the
cumulative ionization and elastic events, the electrons absorbed at the anode
and the field energy must agree within 3 standard errors of their difference,
sqrt(var_gpu / n + var_oracle / n) with n = 16 seeds. Quantities whose
ensemble does not vary (both spreads zero) must be equal.
"""
import json
import os

import numpy as np
import pytest

from paper_2606_05893_gb300 import workloads as W

pytestmark = pytest.mark.gpu

GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "c1_ensemble_1000.json")


def quantities(m):
    return {"count_e": m["count"][0], "count_cu": m["count"][1], "count_ion": m["count"][2],
            "ke_e": m["kinetic"][0], "ke_cu": m["kinetic"][1], "ke_ion": m["kinetic"][2],
            "ionizations": m["n_ionization"], "elastic": m["n_elastic"], "anode_e": m["abs_anode"][0],
            "field_energy": m["field_energy"]}


@pytest.mark.parametrize("precision", [0, 1])
def test_1000_step_ensemble_matches_oracle(precision):
    import torch
    assert torch.cuda.is_available()
    import paper_2606_05893_gb300 as pkg
    gold = json.load(open(GOLD))
    seeds, cps = gold["seeds"], gold["checkpoints"]
    gpu = {cp: [] for cp in cps}
    for seed in seeds:
        sim = pkg.Simulation(W.config_small(seed=seed), precision=precision)
        done = 0
        for cp in cps:
            sim.step(cp - done)
            done = cp
            gpu[cp].append(quantities(sim.moments()))
        sim.close()
    bad = []
    n = len(seeds)
    for cp in cps:
        ref = [quantities(gold["runs"][str(s)][str(cp)]) for s in seeds]
        for k in ref[0]:
            g = np.array([r[k] for r in gpu[cp]], dtype=np.float64)
            o = np.array([r[k] for r in ref], dtype=np.float64)
            se = np.sqrt(g.var(ddof=1) / n + o.var(ddof=1) / n)
            d = abs(g.mean() - o.mean())
            ok = d <= 3 * se if se > 0 else d <= 1e-12 * max(abs(o.mean()), 1e-300)
            if not ok:
                bad.append((cp, k, g.mean(), o.mean(), se))
    assert not bad, bad
