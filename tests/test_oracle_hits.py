"""Pins of the oracle's surface-coupling output: the ions absorbed at the
cathode, for an MD or heat model of the surface (ions that bombard the cathode
are handed over to it: the PIC/MCC paragraph after Eq. 4 and Appendix A). In a field-free box an ion
moves in a straight line, so the step of its crossing, the point where its
path meets z = 0 and its velocity have closed forms; electrons and neutrals
crossing the same plane are not ions and stay out of the log."""
import numpy as np

import oracle as O
from tests._cases import cathode_hits_case


def expected(wl, k, n_steps):
    """Ions crossing within the first n_steps steps: pid (= preload index after
    the electrons and neutrals), crossing step k, crossing point and velocity."""
    xi, vi = wl.preload[2]
    n_before = wl.preload[0][0].shape[0] + wl.preload[1][0].shape[0]
    Lx, Ly, _ = wl.L
    sel = np.nonzero(k < n_steps)[0]
    xc = np.mod(xi[sel, 0] + vi[sel, 0] * (k[sel] + 0.5) * wl.dt, Lx)
    yc = np.mod(xi[sel, 1] + vi[sel, 1] * (k[sel] + 0.5) * wl.dt, Ly)
    pid = (n_before + sel).astype(np.uint32)
    o = np.lexsort((pid, k[sel]))
    return pid[o], k[sel][o], np.column_stack([xc, yc])[o], vi[sel][o]


def test_hit_log_closed_form():
    wl, k = cathode_hits_case()
    ref = O.Oracle(wl)
    ref.step(10)
    h = ref.hits()
    pid, step, xy, v = expected(wl, k, 10)
    assert np.array_equal(h["pid"], pid)
    assert np.array_equal(h["step"], step)
    assert np.all(h["species"] == 2)
    L = max(wl.L)
    assert np.abs(h["xy"] - xy).max() <= 1e-12 * L
    assert np.array_equal(h["v"], v)  # no field: velocities untouched
    # every electron and neutral crossed too, counted but not logged
    m = ref.moments()
    assert m["abs_cathode"][0] == wl.preload[0][0].shape[0]
    assert m["abs_cathode"][1] == wl.preload[1][0].shape[0]
    assert m["abs_cathode"][2] == pid.size


def test_hit_log_empties_and_continues():
    wl, k = cathode_hits_case(seed=12)
    ref = O.Oracle(wl)
    ref.step(6)
    first = ref.hits()
    assert ref.hits()["pid"].size == 0  # read once
    ref.step(6)
    second = ref.hits()
    pid, step, _, _ = expected(wl, k, 12)
    both = np.concatenate([first["pid"], second["pid"]])
    assert np.array_equal(both, pid)
    assert np.all(first["step"] < 6) and np.all(second["step"] >= 6)
