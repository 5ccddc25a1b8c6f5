"""Pins of the oracle's charge exchange: resonant Cu+ + Cu, one of the MCC
collisions the paper lists (the PIC/MCC paragraph with Eq. 4), read as the ion
taking an electron from a neutral of its own element, both keeping x^{n+1} and
v^{n+1/2} (a fast neutral and a slow ion come out). The test of Eq. (4) is the
electrons' one with the ion as projectile: u the ion speed, E = m_ion u^2 / 2,
target density from the neutrals of the ion's cell at x^n. Victims follow the
ionization rule: per cell, events of every channel in order of primary pid take
the neutrals in increasing (Philox victim key, pid); events left without a
neutral are suppressed.

1. Rate: against a fixed background the events per step are Binomial(N, P) with
   P = 1 - exp(-n sigma(E) u dt), sigma taken at the ion's energy (a table
   whose value at the electron-mass energy would be 50 times smaller).
2. Which events succeed, with P = 1: per cell min(ions, neutrals) exchanges, the
   lowest ion pids, the victims with the smallest keys (computed here from the
   Philox generator, pinned to cuRAND elsewhere); the converted particles carry
   exactly the state a run without the channel gives them, everything else is
   untouched, counts per species and the total momentum are unchanged.
3. With electrons ionizing in the same cells, both channels share one victim
   pool in primary-pid order (electron pids come first in the preload).
4. In a plasma run with field, sources and sorting, the per-species counts move
   only by injection, absorption and ionization, and pids stay unique.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2606_05893_gb300 import workloads as W
from tests._cases import bare, cx_cells_case, cx_xsec, isotropic


def _cell(wl, x):
    c = np.floor(x / wl.h).astype(np.int64)
    return (c[:, 2] * wl.ny + c[:, 1]) * wl.nx + c[:, 0]


def _by_pid(o, sp):
    x, v, pid = o.particles(sp)
    return {int(p): (x[k], v[k]) for k, p in enumerate(pid)}


def test_rate_against_background_uses_the_ion_energy():
    n, E_i = 4000, 50.0
    u = math.sqrt(2.0 * E_i * W.E_CHARGE / W.M_CU)
    table_E, table_s = [1.0, 100.0], [1e-19, 1e-17]
    sigma = 1e-19 + (E_i - 1.0) / 99.0 * (1e-17 - 1e-19)
    dt = 1e-14
    n0 = 0.5 / (u * sigma * dt)  # P = 1 - e^-0.5
    wl = bare(nx=8, ny=8, nz=8, h=1e-8, dt=dt, weight=1e-30, xsec=[cx_xsec(table_s, E=table_E)], seed=4)
    rng = np.random.default_rng(4)
    L = np.array(wl.L)
    x = (0.25 + 0.5 * rng.random((n, 3))) * L
    wl.preload = [(np.zeros((0, 3)), np.zeros((0, 3))), (np.zeros((0, 3)), np.zeros((0, 3))),
                  (x, isotropic(rng, n, u))]
    o = O.Oracle(wl, background_density=n0)
    steps = 3
    o.step(steps)
    P = -math.expm1(-0.5)
    N = n * steps
    m = o.moments()
    assert abs(m["n_cx"] - N * P) < 5 * math.sqrt(N * P * (1 - P)), (m["n_cx"], N * P)
    assert m["n_ionization"] == 0 and m["n_elastic"] == 0
    assert m["count"] == [0, 0, n]  # a fixed background converts nothing


def _expected(wl, seed_key, step, with_electrons):
    """Per cell: events (electrons with lower pids first, then ions) in pid order,
    victims by (key, pid); returns the successful (primary pid, victim pid) pairs
    and the number suppressed."""
    (xe, _), (xn, _), (xi, _) = wl.preload
    ne, nn = xe.shape[0], xn.shape[0]
    pe = np.arange(ne)
    pn = np.arange(ne, ne + nn)
    pi = np.arange(ne + nn, ne + nn + xi.shape[0])
    ce, cn, ci = _cell(wl, xe), _cell(wl, xn), _cell(wl, xi)
    key = [seed_key & 0xFFFFFFFF, seed_key >> 32]
    pairs, supp = [], 0
    for c in np.unique(np.concatenate([ce, ci])):
        vic = pn[cn == c]
        if vic.size == 0:
            continue  # no target density: no event
        ev = np.sort(np.concatenate([pe[ce == c] if with_electrons else [], pi[ci == c]]).astype(np.int64))
        keys = [(int(O.philox([int(p), step, 32, 0], key)[0]) << 32) | int(p) for p in vic]
        order = [int(vic[k]) for k in np.argsort(keys)]
        for r, p in enumerate(ev):
            if r < len(order):
                pairs.append((int(p), order[r]))
            else:
                supp += 1
    return pairs, supp, ne


def test_exchanges_take_the_lowest_pids_and_smallest_keys():
    wl = cx_cells_case()
    base = cx_cells_case()
    base.xsec = []
    o, ob = O.Oracle(wl, cg_rtol=1e-13), O.Oracle(base, cg_rtol=1e-13)
    m0 = o.moments()
    o.step()
    ob.step()
    m = o.moments()
    pairs, supp, _ = _expected(wl, wl.seed, 0, False)
    assert len(pairs) == 60 + 7 and supp == 63  # the four cells of the case
    assert m["n_cx"] == len(pairs) and m["n_suppressed"] == supp and m["n_ionization"] == 0
    assert m["count"] == m0["count"]
    ions, neut = _by_pid(o, 2), _by_pid(o, 1)
    ions_b, neut_b = _by_pid(ob, 2), _by_pid(ob, 1)
    swapped_ions = {p for p, _ in pairs}
    victims = {v for _, v in pairs}
    assert set(ions) == (set(ions_b) - swapped_ions) | victims
    assert set(neut) == (set(neut_b) - victims) | swapped_ions
    for p in ions:  # victims now ions with the state the neutral run gives them
        ref = neut_b[p] if p in victims else ions_b[p]
        assert np.array_equal(ions[p][0], ref[0]) and np.array_equal(ions[p][1], ref[1])
    for p in neut:
        ref = ions_b[p] if p in swapped_ions else neut_b[p]
        assert np.array_equal(neut[p][0], ref[0]) and np.array_equal(neut[p][1], ref[1])
    # momentum of the heavy particles is only moved between species
    mom = lambda d: np.sum([v for _, v in d.values()], axis=0)
    assert np.allclose(mom(ions) + mom(neut), mom(ions_b) + mom(neut_b), rtol=1e-13, atol=0)


def test_ionization_and_exchange_share_the_victims():
    wl = cx_cells_case(sigma_ion=1e-10, with_electrons=True)
    o = O.Oracle(wl, cg_rtol=1e-13)
    m0 = o.moments()
    o.step()
    m = o.moments()
    pairs, supp, ne = _expected(wl, wl.seed, 0, True)
    n_ion = sum(1 for p, _ in pairs if p < ne)
    n_cx = len(pairs) - n_ion
    # dense cell: 25 e + 60 ions on 90 neutrals, all succeed; (5,5,5): 25 e + 70
    # ions on 7 neutrals, the 7 lowest pids (electrons) win; no neutrals in (1,6,2)
    assert (n_ion, n_cx, supp) == (25 + 7, 60, 25 + 70 - 7)
    assert m["n_ionization"] == n_ion and m["n_cx"] == n_cx and m["n_suppressed"] == supp
    log = o.ionization_log()
    assert sorted((int(a), int(b)) for a, b, _ in log) == sorted((p, v) for p, v in pairs if p < ne)
    # ionizations add an electron and an ion and remove a neutral; exchanges move
    # one ion to the neutrals and one neutral to the ions
    c0 = m0["count"]
    assert m["count"] == [c0[0] + n_ion, c0[1] - n_ion, c0[2] + n_ion]
    neut = _by_pid(o, 1)
    assert {p for p, _ in pairs if p >= ne} <= set(neut)


def test_bookkeeping_in_a_plasma_run_with_exchange():
    # counts per species move only by injection, absorption and ionization
    # (an exchange turns one ion into a neutral and one neutral into an ion);
    # pids stay unique across species
    wl = W.config_small(seed=47, n_preload=4000)
    wl.xsec = list(wl.xsec) + [cx_xsec(1e-16)]
    o = O.Oracle(wl, cg_rtol=1e-10)
    m = o.moments()
    cx_seen = 0
    for _ in range(12):
        o.step()
        m1 = o.moments()
        d_inj = [a - b for a, b in zip(m1["injected"], m["injected"])]
        d_abs = [a + c - b - d for a, b, c, d in zip(m1["abs_cathode"], m["abs_cathode"], m1["abs_anode"], m["abs_anode"])]
        d_ion = m1["n_ionization"] - m["n_ionization"]
        expect = [m["count"][0] + d_inj[0] - d_abs[0] + d_ion,
                  m["count"][1] + d_inj[1] - d_abs[1] - d_ion,
                  m["count"][2] + d_inj[2] - d_abs[2] + d_ion]
        assert m1["count"] == expect
        cx_seen += m1["n_cx"] - m["n_cx"]
        pids = np.concatenate([o.particles(sp)[2] for sp in range(3)])
        assert np.unique(pids).size == pids.size
        m = m1
    assert cx_seen > 0
