"""Pins of the oracle's injection (superparticles injected from the cathode,
PIC/MCC paragraph), cell sort, moments and the integer bookkeeping of a step.

- Injection: integer counts follow the carry accumulator of the expected count
  mu = flux pi R^2 dt / w; positions are uniform on the disk (<r^2> = R^2/2);
  velocities are half-Maxwellian (<vz> = s sqrt(2/pi), <vx^2> = s^2).
- Sort: the order equals numpy's lexsort by (cell, pid), cell offsets equal the
  prefix sums of numpy's bincount.
- Moments: parallel-plate field energy eps0 E^2 V / 2 for the vacuum solution;
  kinetic energy against math.fsum.
- Conservation: N^{n+1} = N^n + injected - absorbed +- ionizations, per species.
"""
import math

import numpy as np
import pytest
from scipy import stats

import oracle as O
from paper_2606_05893_gb300 import workloads as W
from tests._cases import bare


def _source_case(mu, R=20e-9, T=5800.0, species=0, weight=1.0):
    wl = bare(nx=16, ny=16, nz=16, h=5e-9, dt=1e-16, weight=weight)
    L = wl.L
    area = math.pi * R * R
    flux = mu * weight / (area * wl.dt)
    wl.sources = [W.Source(species, L[0] / 2, L[1] / 2, R, flux, T)]
    return wl


def test_injection_counts_follow_carry_accumulator():
    mu = 0.3719
    wl = _source_case(mu)
    o = O.Oracle(wl)
    total = 0
    for n in range(1, 200):
        total += o.inject()
        o.step_index = n
        assert total in (math.floor(n * mu) - 1, math.floor(n * mu))
    assert total == math.floor(199 * mu)


def test_injection_disk_and_half_maxwellian():
    mu, R, T = 200_000.4, 20e-9, 5800.0
    wl = _source_case(mu, R, T)
    o = O.Oracle(wl)
    n = o.inject()
    assert n == 200_000
    x, v, pid = o.particles(0)
    assert np.array_equal(pid, np.arange(n, dtype=np.uint32))
    L = wl.L
    r2 = (x[:, 0] - L[0] / 2) ** 2 + (x[:, 1] - L[1] / 2) ** 2
    assert stats.kstest(r2 / R ** 2, "uniform").pvalue > 1e-3
    th = np.arctan2(x[:, 1] - L[1] / 2, x[:, 0] - L[0] / 2)
    assert stats.kstest((th + math.pi) / (2 * math.pi), "uniform").pvalue > 1e-3
    s = math.sqrt(W.K_B * T / W.M_E)
    assert abs(v[:, 0].mean()) < 5 * s / math.sqrt(n)
    assert abs((v[:, 0] ** 2).mean() / s ** 2 - 1) < 5 * math.sqrt(2 / n)
    assert abs((v[:, 1] ** 2).mean() / s ** 2 - 1) < 5 * math.sqrt(2 / n)
    assert np.all(v[:, 2] > 0)
    mvz = s * math.sqrt(2 / math.pi)
    assert abs(v[:, 2].mean() - mvz) < 5 * s * math.sqrt(1 - 2 / math.pi) / math.sqrt(n)
    assert stats.kstest(v[:, 0] / s, "norm").pvalue > 1e-3
    # first partial step z = U vz dt
    assert np.all((x[:, 2] >= 0) & (x[:, 2] <= v[:, 2] * wl.dt))
    assert abs(x[:, 2].mean() - 0.5 * mvz * wl.dt) < 5 * 0.6 * s * wl.dt / math.sqrt(n)


def test_sort_matches_lexsort_and_bincount():
    wl = W.config_tiny()
    o = O.Oracle(wl)
    o.sort()
    h = wl.h
    for sp in range(3):
        x, v, pid = o.particles(sp)
        inv = 1.0 / h
        i = np.minimum(np.floor(x[:, 0] * inv).astype(np.int64), wl.nx - 1)
        j = np.minimum(np.floor(x[:, 1] * inv).astype(np.int64), wl.ny - 1)
        k = np.minimum(np.floor(x[:, 2] * inv).astype(np.int64), wl.nz - 1)
        cell = (k * wl.ny + j) * wl.nx + i
        order = np.lexsort((pid, cell))
        assert np.array_equal(order, np.arange(pid.size))
        cs = o.cell_start(sp)
        ref = np.concatenate([[0], np.cumsum(np.bincount(cell, minlength=wl.nx * wl.ny * wl.nz))])
        assert np.array_equal(cs, ref)


def test_vacuum_field_energy_is_parallel_plate():
    wl = bare(nx=6, ny=5, nz=12, h=4e-9, phi_c=0.0, phi_a=500.0)
    o = O.Oracle(wl, cg_rtol=1e-14)
    o.step()
    m = o.moments()
    L = wl.L
    E = 500.0 / L[2]
    assert m["field_energy"] == pytest.approx(0.5 * W.EPS0 * E * E * L[0] * L[1] * L[2], rel=1e-12)


def test_kinetic_energy_and_charge_vs_fsum():
    wl = W.config_tiny()
    o = O.Oracle(wl)
    m = o.moments()
    for sp in range(3):
        x, v, pid = o.particles(sp)
        s = wl.species[sp]
        ke = 0.5 * s.mass_kg * s.weight * math.fsum((v * v).reshape(-1))
        assert m["kinetic"][sp] == pytest.approx(ke, rel=1e-13)
    q = math.fsum(s.charge_C * s.weight * len(o.particles(i)[2]) for i, s in enumerate(wl.species))
    assert m["total_charge"] == pytest.approx(q, rel=1e-14, abs=1e-40)


def test_particle_bookkeeping_over_steps():
    wl = W.config_small(n_preload=4000)
    o = O.Oracle(wl)
    pre = [p[0].shape[0] for p in wl.preload]
    o.step(12)
    m = o.moments()
    ion = m["n_ionization"]
    e, n, i = m["count"]
    assert e == pre[0] + m["injected"][0] - m["abs_cathode"][0] - m["abs_anode"][0] + ion
    assert n == pre[1] + m["injected"][1] - m["abs_cathode"][1] - m["abs_anode"][1] - ion
    assert i == pre[2] + m["injected"][2] - m["abs_cathode"][2] - m["abs_anode"][2] + ion
    # pids stay unique
    allp = np.concatenate([o.particles(s)[2] for s in range(3)])
    assert np.unique(allp).size == allp.size
    assert m["next_pid"] == sum(pre) + sum(m["injected"]) + ion
