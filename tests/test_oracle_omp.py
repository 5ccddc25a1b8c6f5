"""The OpenMP build of the oracle (the same source compiled with -fopenmp, used
as the CPU baseline on all host cores) gives results bit-identical to the
serial build with any number of threads: every sum keeps one fixed order
(chunked dot products in both builds, the push's bookkeeping in particle
order), so parallel execution changes no rounding. Checked on the 32x32x64
workload (MCC, ionization and injection active) and on one with charge
exchange, over enough steps for collisions, absorption and a cell sort.
"""
import numpy as np
import pytest

import oracle
from paper_2606_05893_gb300 import workloads as W


def _state(wl, steps, omp, threads):
    if omp:
        oracle.set_threads(threads)
    o = oracle.Oracle(wl, omp=omp)
    o.step(steps)
    out = {"phi": o.phi(), "rho": o.rho(), "log": o.ionization_log(), "moments": o.moments(),
           "particles": [o.particles(s) for s in range(len(wl.species))]}
    o.close()
    return out


def _identical(a, b):
    for k in ("phi", "rho", "log"):
        if not np.array_equal(a[k], b[k]):
            return k
    for s, (pa, pb) in enumerate(zip(a["particles"], b["particles"])):
        for x, y in zip(pa, pb):
            if not np.array_equal(x, y):
                return f"particles of species {s}"
    for k, v in a["moments"].items():
        if not np.array_equal(np.asarray(v), np.asarray(b["moments"][k])):
            return f"moment {k}"
    return None


@pytest.mark.parametrize("cx", [False, True])
def test_openmp_build_bit_identical(cx):
    wl = W.config_small(seed=5)
    if cx:  # resonant charge exchange Cu+ + Cu at a constant cross-section
        wl.xsec = list(wl.xsec) + [W.XSec(W.XS_CHARGE_EXCHANGE, 2, 1, 1, 0.0, np.array([1.0]), np.array([2e-18]))]
    steps = 45  # two cell sorts (interval 20), ionizations and absorptions
    ref = _state(wl, steps, False, 1)
    assert sum(ref["moments"]["abs_anode"]) + sum(ref["moments"]["abs_cathode"]) > 0
    assert ref["moments"]["n_ionization"] > 0 and ref["moments"]["n_elastic"] > 0
    if cx:
        assert ref["moments"]["n_cx"] > 0
    for threads in (1, 2, 4):
        got = _state(wl, steps, True, threads)
        assert _identical(ref, got) is None, (threads, _identical(ref, got))
    oracle.set_threads(0)


def test_set_threads_reports_count():
    assert oracle.set_threads(2) == 2
    assert oracle.set_threads(0) >= 1
    assert oracle.lib().or_set_threads(4) == 1  # the serial build always runs one thread
