"""Autotuner of the per-instance launch parameters for handles that hold several
instances: the cell-sort interval and the launch shape (thread blocks per SM)
of the particle kernels.

The cell sort (a2) only reorders particles; it costs a pass over the stores
and buys locality for the deposit atomics and the field gathers, which decays
as particles move. The grid of the particle kernels trades occupancy against
the rounds of the block-level compaction. The best pair depends on each
instance's grid, particle count and speeds.

Every candidate pair is timed from the same state: each instance is
checkpointed first (pic_save) and restored (pic_load) before every candidate,
sorted at once (so every candidate starts from the same order), and then all
instances run one common period of the candidate intervals (their least common
multiple, 40 steps for 5, 10, 20, 40: each interval pays exactly its share of
sorts) with per-phase CUDA-event timing on; each instance keeps the pair with
the lowest device time per step. The instances are restored once more at the
end, so tuning leaves the run where it was. Choices are cached per (grid, particle-count bucket): a later call finds
the instances whose bucket is cached and tunes only the others.
"""
from __future__ import annotations

import math
import os
from functools import reduce
import shutil
import tempfile

from . import pic_get_phase_times, pic_set_launch_shape, pic_set_profiling, pic_set_sort_interval, pic_sort_now

INTERVALS = (5, 10, 20, 40)
SHAPES = (4, 8, 16)
_CACHE = {}


def bucket(wl, n_particles):
    """Cache key: the grid and the particle count rounded to a power of two."""
    return (wl.nx, wl.ny, wl.nz, int(round(math.log2(max(n_particles, 1)))))


def _tmpdir():
    base = "/dev/shm" if os.path.isdir("/dev/shm") and os.access("/dev/shm", os.W_OK) else None
    return tempfile.mkdtemp(prefix="pic_tune_", dir=base)


def tune(sim, intervals=INTERVALS, shapes=SHAPES, window=None, cache=_CACHE):
    """Pick (sort interval, blocks per SM) for every instance of `sim`. The window
    defaults to the least common multiple of the intervals. Returns the chosen
    pairs and {(interval, shape): [ms per step per instance]} (None where an
    instance's choice came from the cache)."""
    n_inst = len(sim.wls)
    if window is None:
        window = reduce(lambda a, b: a * b // math.gcd(a, b), intervals)
    counts = [sum(sim.count(sp, i) for sp in range(len(sim.wls[i].species))) for i in range(n_inst)]
    keys = [bucket(sim.wls[i], counts[i]) for i in range(n_inst)]
    todo = [i for i in range(n_inst) if keys[i] not in cache]
    measured = {}
    if todo:
        d = _tmpdir()
        try:
            paths = {i: os.path.join(d, f"inst{i}.ckpt") for i in range(n_inst)}
            for i in range(n_inst):
                sim.save(paths[i], inst=i)
            for iv in intervals:
                for sh in shapes:
                    for i in range(n_inst):
                        sim.load(paths[i], inst=i)
                        pic_set_sort_interval(sim.h, i, iv)
                        pic_set_launch_shape(sim.h, i, sh)
                        pic_sort_now(sim.h, i)
                    pic_set_profiling(sim.h, True)
                    sim.step(window)
                    per = []
                    for i in range(n_inst):
                        phases = pic_get_phase_times(sim.h, i)
                        per.append(sum(ms for ms, _ in phases.values()) / window if i in todo else None)
                    pic_set_profiling(sim.h, False)
                    measured[(iv, sh)] = per
            for i in range(n_inst):
                sim.load(paths[i], inst=i)
        finally:
            shutil.rmtree(d, ignore_errors=True)
        # per bucket: the pair with the least summed time over its instances
        for k in {keys[i] for i in todo}:
            members = [i for i in todo if keys[i] == k]
            cache[k] = min(measured, key=lambda c: sum(measured[c][i] for i in members))
    chosen = []
    for i in range(n_inst):
        iv, sh = cache[keys[i]]
        pic_set_sort_interval(sim.h, i, iv)
        pic_set_launch_shape(sim.h, i, sh)
        chosen.append((iv, sh))
    return chosen, measured


def tune_sort_interval(sim, candidates=INTERVALS, window=None):
    """The sort interval alone (launch shape kept at 8 blocks per SM)."""
    chosen, measured = tune(sim, intervals=candidates, shapes=(8,), window=window, cache={})
    return [c[0] for c in chosen], {iv: measured[(iv, 8)] for iv in candidates}
