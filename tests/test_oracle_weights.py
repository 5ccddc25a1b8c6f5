"""Pins of variable-weight particles (integer multiplicities) in the oracle.

A particle of multiplicity m stands for m x (species weight) physical particles:
it deposits m times the charge, counts m times as an MCC target, and an event
between a primary of multiplicity mp and a victim of multiplicity mv moves
ms = min(mp, mv): the partner holding more keeps the rest in place, the part
that changes species becomes a new particle of multiplicity ms, and a primary
electron that moves only part of itself loses the ionization energy with
probability ms / mp.

1. Multiplicities 1 with variable weights on give the plain rule's particles
   and counts.
2. A uniform multiplicity k at weight w gives what weight k w gives (charge,
   fields, trajectories, events).
3. With unequal multiplicities and no particle leaving the box, the heavy
   particles (neutrals + ions) and the net charge (electrons - ions) are
   conserved exactly in multiplicity units, pids stay unique, 3 pids are taken
   per successful event, and partial conversions leave neutrals alive with a
   lower multiplicity.
4. Primaries of multiplicity 4 ionizing victims of multiplicity 1 lose energy
   in a quarter of the events (binomial bound).
5. Charge exchange and ionization together with unequal multiplicities keep
   the same invariants.
6. In a field-free box, where every particle crosses the cathode at a known
   step, the absorbed energy and the charge collected in a step are the closed
   sums over the crossing particles weighted by their multiplicities, and the
   absorbed counts stay counts of superparticles.
"""
import math

import numpy as np

import oracle as O
from tests._cases import cx_cells_case, ionization_cells_case, weighted_ionization_case, with_multiplicities


def _by_pid(o, sp):
    x, v, pid = o.particles(sp)
    m = o.multiplicity(sp)
    order = np.argsort(pid)
    return x[order], v[order], pid[order], m[order]


def test_unit_multiplicities_match_plain_rule():
    plain = ionization_cells_case(seed=4)
    unit = ionization_cells_case(seed=4)
    unit.variable_weights = True
    unit.preload = [(x, v, np.ones(x.shape[0], dtype=np.uint32)) for x, v in unit.preload]
    a, b = O.Oracle(plain, cg_rtol=1e-13), O.Oracle(unit, cg_rtol=1e-13)
    a.step(1)
    b.step(1)
    ma, mb = a.moments(), b.moments()
    assert ma["n_ionization"] > 20
    for k in ("count", "n_ionization", "n_elastic", "n_suppressed", "abs_cathode", "abs_anode"):
        assert ma[k] == mb[k], k
    for sp in range(3):
        xa, va, pa, _ = _by_pid(a, sp)
        xb, vb, pb, mb_ = _by_pid(b, sp)
        assert np.array_equal(pa, pb)
        assert np.array_equal(xa, xb) and np.array_equal(va, vb)
        assert np.all(mb_ == 1)
    # the weighted rule reserves 3 pids per successful event, the plain one 1 per ionization
    n0 = sum(x.shape[0] for x, _ in plain.preload)
    assert ma["next_pid"] == n0 + ma["n_ionization"]
    assert mb["next_pid"] == n0 + 3 * mb["n_ionization"]
    a.close()
    b.close()


def test_uniform_multiplicity_equals_scaled_weight():
    k = 3
    scaled = ionization_cells_case(seed=6)
    for s in scaled.species:
        s.weight *= k
    mult = ionization_cells_case(seed=6)
    mult.variable_weights = True
    mult.preload = [(x, v, np.full(x.shape[0], k, dtype=np.uint32)) for x, v in mult.preload]
    a, b = O.Oracle(scaled, cg_rtol=1e-13), O.Oracle(mult, cg_rtol=1e-13)
    a.step(1)
    b.step(1)
    ma, mb = a.moments(), b.moments()
    assert ma["n_ionization"] > 20
    for key in ("count", "n_ionization", "n_elastic", "n_suppressed"):
        assert ma[key] == mb[key], key
    assert math.isclose(ma["total_charge"], mb["total_charge"], rel_tol=1e-12, abs_tol=1e-30)
    for sp in range(3):
        assert math.isclose(ma["kinetic"][sp], mb["kinetic"][sp], rel_tol=1e-12)
        xa, va, pa, _ = _by_pid(a, sp)
        xb, vb, pb, mm = _by_pid(b, sp)
        assert np.array_equal(pa, pb)
        assert np.all(mm == k)
        assert np.abs(xa - xb).max(initial=0.0) <= 1e-12 * max(scaled.L)
        assert np.abs(va - vb).max(initial=0.0) <= 1e-10 * np.abs(va).max(initial=1.0)
    # the preload is charge-neutral (electrons on ions), so rho is a rounding
    # residue: compare against one particle's charge density
    ra, rb = a.rho(), b.rho()
    one = abs(scaled.species[0].charge_C) * scaled.species[0].weight / scaled.h ** 3
    assert np.abs(ra - rb).max() <= 1e-12 * one
    a.close()
    b.close()


def test_invariants_with_unequal_multiplicities():
    wl = weighted_ionization_case(seed=8)
    o = O.Oracle(wl, cg_rtol=1e-13)

    def totals():
        return [int(o.multiplicity(sp).astype(np.int64).sum()) for sp in range(3)]

    e0, n0, i0 = totals()
    pid0 = o.moments()["next_pid"]
    q0 = o.moments()["total_charge"]
    partial = False
    for _ in range(3):
        before = o.moments()
        o.step(1)
        after = o.moments()
        e, n, i = totals()
        assert after["abs_cathode"] == [0, 0, 0] and after["abs_anode"] == [0, 0, 0]
        assert n + i == n0 + i0          # heavy particles
        assert e - i == e0 - i0          # net charge in multiplicity units
        ns = (after["n_ionization"] - before["n_ionization"]) + (after["n_cx"] - before["n_cx"])
        assert after["next_pid"] - before["next_pid"] == 3 * ns
        pids = np.concatenate([o.particles(sp)[2] for sp in range(3)])
        assert np.unique(pids).size == pids.size
        mn = o.multiplicity(1)
        partial = partial or bool(np.any(mn < wl.preload[1][2].max()))
    assert o.moments()["n_ionization"] > 20
    assert partial
    assert math.isclose(o.moments()["total_charge"], q0, rel_tol=1e-12, abs_tol=1e-25)
    assert o.moments()["next_pid"] > pid0
    o.close()


def test_primary_energy_loss_probability():
    # primaries of multiplicity 4 against victims of multiplicity 1: each event
    # moves 1 of 4, so the primary loses the ionization energy with probability 1/4
    wl = weighted_ionization_case(seed=9, m_e=(4, 4), m_n=(1, 1), n_dense_e=1500, n_dense_n=4000)
    o = O.Oracle(wl, cg_rtol=1e-13)
    x0, v0, p0, _ = _by_pid(o, 0)
    o.step(1)
    log = o.ionization_log()
    assert log.shape[0] > 200
    prim = np.unique(log[:, 0])
    x1, v1, p1, m1 = _by_pid(o, 0)
    idx0 = np.searchsorted(p0, prim)
    idx1 = np.searchsorted(p1, prim)
    s0 = np.linalg.norm(v0[idx0], axis=1)
    s1 = np.linalg.norm(v1[idx1], axis=1)
    lost = s1 < 0.99 * s0   # an ionization takes at least 7.73 of 100 eV: 4 % of the speed
    n = prim.size
    frac = lost.mean()
    sd = math.sqrt(0.25 * 0.75 / n)
    assert abs(frac - 0.25) < 4 * sd, (frac, n)
    # each event made a secondary of multiplicity 1 (the part moved)
    sec = np.setdiff1d(p1, p0)
    msec = m1[np.searchsorted(p1, sec)]
    assert np.all(msec == 1)
    o.close()


def test_exchange_and_ionization_invariants_with_unequal_multiplicities():
    wl = with_multiplicities(cx_cells_case(sigma_ion=1e-10, with_electrons=True), 1, 5, seed=12)
    o = O.Oracle(wl, cg_rtol=1e-13)

    def totals():
        return [int(o.multiplicity(sp).astype(np.int64).sum()) for sp in range(3)]

    e0, n0, i0 = totals()
    before = o.moments()
    o.step(1)
    m = o.moments()
    e, n, i = totals()
    assert m["abs_cathode"] == [0, 0, 0] and m["abs_anode"] == [0, 0, 0]
    assert m["n_cx"] > 20 and m["n_ionization"] > 10
    assert n + i == n0 + i0
    assert e - i == e0 - i0
    ns = m["n_ionization"] + m["n_cx"]
    assert m["next_pid"] - before["next_pid"] == 3 * ns
    pids = np.concatenate([o.particles(sp)[2] for sp in range(3)])
    assert np.unique(pids).size == pids.size
    o.close()


def test_weighted_absorption_closed_form():
    # field-free box (weight 1e-30, both electrodes at 0 V): every particle moves
    # in a straight line and crosses the cathode at a known step. Absorbed counts
    # stay counts of superparticles; the absorbed energy sums (1/2) m w mw |v|^2
    # and the charge collected in a step q w mw over the particles crossing in it
    from tests._cases import cathode_hits_case
    wl, k = cathode_hits_case()
    wl = with_multiplicities(wl, 1, 7, seed=21)
    (xe, ve, me), (xn, vn, mn), (xi, vi, mi) = wl.preload
    o = O.Oracle(wl)
    s_chk = 5
    o.step(s_chk)
    before = o.moments()
    o.step(1)  # step s_chk: only the ions with k == s_chk cross
    m = o.moments()
    sel = k == s_chk
    assert sel.sum() > 0
    qi = wl.species[2].charge_C * wl.species[2].weight
    assert math.isclose(m["charge_to_cathode_last"], qi * float(mi[sel].sum()), rel_tol=1e-14)
    o.step(20)
    m = o.moments()
    assert m["abs_cathode"] == [xe.shape[0], xn.shape[0], xi.shape[0]]
    for sp, (v, mw) in enumerate([(ve, me), (vn, mn), (vi, mi)]):
        s = wl.species[sp]
        want = 0.5 * s.mass_kg * s.weight * float(np.sum(mw * np.sum(v * v, axis=1)))
        assert math.isclose(m["abs_energy_cathode"][sp], want, rel_tol=1e-12), sp
    assert m["total_charge"] == 0.0 and m["count"] == [0, 0, 0]
    assert before["abs_cathode"][2] < xi.shape[0]
    o.close()
