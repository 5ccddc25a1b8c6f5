"""Sort-interval autotuner for handles that hold several instances.

The cell sort (a2) only reorders particles; it costs a pass over the stores
and buys locality for the deposit atomics and the field gathers that decays as
particles move. The best interval therefore depends on each instance's grid,
particle count and speeds. For every candidate, all instances run a window of
steps with per-phase CUDA-event timing on; each instance then keeps the
candidate with the lowest device time per step.
"""
from __future__ import annotations

from . import pic_get_phase_times, pic_set_profiling, pic_set_sort_interval

CANDIDATES = (5, 10, 20, 50)


def tune_sort_interval(sim, candidates=CANDIDATES, window=None):
    """Pick the sort interval of every instance of `sim`; returns the chosen
    intervals and the measured ms per step, {candidate: [ms per instance]}."""
    n_inst = len(sim.wls)
    window = window or max(candidates)
    measured = {}
    for cand in candidates:
        for i in range(n_inst):
            pic_set_sort_interval(sim.h, i, cand)
        pic_set_profiling(sim.h, True)
        sim.step(window)
        per = []
        for i in range(n_inst):
            phases = pic_get_phase_times(sim.h, i)
            per.append(sum(ms for ms, _ in phases.values()) / window)
        pic_set_profiling(sim.h, False)
        measured[cand] = per
    chosen = []
    for i in range(n_inst):
        best = min(candidates, key=lambda c: measured[c][i])
        pic_set_sort_interval(sim.h, i, best)
        chosen.append(best)
    return chosen, measured
