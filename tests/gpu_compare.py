"""Comparison helpers for the GPU-vs-oracle parity tests (test code only)."""
import numpy as np


def by_pid(x, v, pid):
    o = np.argsort(pid, kind="stable")
    return x[o], v[o], pid[o]


def periodic_dx(a, b, L):
    d = np.abs(a - b)
    for c in (0, 1):
        d[:, c] = np.minimum(d[:, c], L[c] - d[:, c])
    return d


def compare_particles(sim, ref, wl, sp, tol_x, tol_v, inst=0):
    """Match particles by pid; return (max |dx| / L, max |dv| / max|v|)."""
    xg, vg, pg = by_pid(*sim.particles(sp, inst))
    xo, vo, po = by_pid(*ref.particles(sp))
    assert pg.size == po.size, (sp, pg.size, po.size)
    assert np.array_equal(pg, po), f"species {sp}: pid sets differ"
    if pg.size == 0:
        return 0.0, 0.0
    L = np.array(wl.L)
    ex = (periodic_dx(xg, xo, L) / L.max()).max()
    vmax = np.abs(vo).max()
    ev = np.abs(vg - vo).max() / vmax if vmax > 0 else 0.0
    assert ex <= tol_x, f"species {sp}: position error {ex:.3e} > {tol_x:.1e}"
    assert ev <= tol_v, f"species {sp}: velocity error {ev:.3e} > {tol_v:.1e}"
    return ex, ev


def rel_inf(a, b):
    s = np.abs(b).max()
    return np.abs(a - b).max() / (s if s > 0 else 1.0)


INT_KEYS = ("count", "injected", "abs_cathode", "abs_anode", "n_ionization", "n_elastic", "n_suppressed",
            "n_cx", "next_pid")


def compare_integer_moments(mg, mo):
    for k in INT_KEYS:
        assert mg[k] == mo[k], f"{k}: gpu {mg[k]} oracle {mo[k]}"
