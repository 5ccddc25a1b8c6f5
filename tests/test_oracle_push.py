"""Pins of the oracle's field gather and leapfrog push (PIC/MCC paragraph:
superparticles move as a result of electric forces; field from Eq. 1).

1. A uniform applied field with negligible space charge: leapfrog is exact for a
   constant acceleration, x^n = x^0 + n dt v^{-1/2} + a dt^2 n(n+1)/2.
2. Cold-plasma oscillation in a periodic direction: the measured frequency equals
   the leapfrog dispersion relation sin(w dt/2) = W dt/2, with W the plasma
   frequency times the cos(kh/2) factor of the cloud-in-cell/finite-difference
   grid (derived for particles loaded at cell centres), and the total energy
   stays bounded.
"""
import math

import numpy as np

import oracle as O
from paper_2606_05893_gb300 import workloads as W
from tests._cases import bare


def test_uniform_field_trajectory_is_exact():
    wl = bare(nx=4, ny=4, nz=16, h=5e-9, dt=1e-16, phi_c=0.0, phi_a=100.0, weight=1e-30)
    rng = np.random.default_rng(1)
    L = np.array(wl.L)
    n = 50
    x0 = rng.random((n, 3)) * L * np.array([1, 1, 0.3]) + np.array([0, 0, 0.2 * L[2]])
    v0 = rng.standard_normal((n, 3)) * 1e5
    wl.preload = [(x0, v0), (np.zeros((0, 3)), np.zeros((0, 3))), (x0.copy(), -v0)]
    o = O.Oracle(wl, cg_rtol=1e-14)
    Ez = -(wl.phi_anode - wl.phi_cathode) / L[2]
    steps = 40
    o.step(steps)
    for sp in (0, 2):
        s = wl.species[sp]
        a = s.charge_C / s.mass_kg * Ez
        x, v, pid = o.particles(sp)
        order = np.argsort(pid)
        x, v = x[order], v[order]
        base = 0 if sp == 0 else n
        assert np.array_equal(np.sort(pid), np.arange(base, base + n, dtype=np.uint32))
        xin, vin = wl.preload[sp]
        N = steps
        ez = xin[:, 2] + N * wl.dt * vin[:, 2] + a * wl.dt ** 2 * N * (N + 1) / 2
        ex = np.mod(xin[:, :2] + N * wl.dt * vin[:, :2], L[:2])
        assert np.allclose(x[:, 2], ez, rtol=0, atol=1e-12 * L[2])
        d = np.abs(x[:, :2] - ex)
        d = np.minimum(d, L[:2] - d)
        assert d.max() <= 1e-12 * L[0]
        assert np.allclose(v[:, 2], vin[:, 2] + a * wl.dt * N, rtol=1e-12, atol=1e-12 * abs(a * wl.dt * N))
        assert np.allclose(v[:, :2], vin[:, :2], rtol=1e-14, atol=0)


def cold_plasma_case(nx=16, ny=2, nz=128, h=1e-8, dt=1e-16, wpe_dt=0.2, amp=1e-3):
    wpe = wpe_dt / dt
    n0 = wpe ** 2 * W.EPS0 * W.M_E / W.E_CHARGE ** 2
    w = n0 * h ** 3
    wl = bare(nx=nx, ny=ny, nz=nz, h=h, dt=dt, weight=w, rho_background=W.E_CHARGE * n0, cg_rtol=1e-13)
    g = np.stack(np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij"), -1).reshape(-1, 3)
    x0 = (g + 0.5) * h
    k = 2 * math.pi / (nx * h)
    x = x0.copy()
    x[:, 0] += amp * h * np.sin(k * x0[:, 0])
    wl.preload = [(x, np.zeros_like(x)), (np.zeros((0, 3)), np.zeros((0, 3))), (np.zeros((0, 3)), np.zeros((0, 3)))]
    return wl, x0, k, wpe


def test_cold_plasma_oscillation_frequency_and_energy():
    wl, x0, k, wpe = cold_plasma_case()
    o = O.Oracle(wl, cg_rtol=1e-13)
    Lz = wl.L[2]
    mid = (x0[:, 2] > Lz / 4) & (x0[:, 2] < 3 * Lz / 4)
    s = np.sin(k * x0[:, 0])
    amps, kin, fld = [], [], []
    for n in range(160):
        x, v, pid = o.particles(0)
        xo = x[np.argsort(pid)]
        xi = xo[:, 0] - x0[:, 0]
        amps.append(np.sum(xi[mid] * s[mid]) / np.sum(s[mid] ** 2))
        o.step()
        m = o.moments()
        kin.append(m["kinetic"][0])   # at t^{n+1/2}
        fld.append(m["field_energy"])  # at t^n
    a = np.array(amps)
    c = np.sum(a[1:-1] * (a[2:] + a[:-2])) / (2 * np.sum(a[1:-1] ** 2))
    w_meas = math.acos(c) / wl.dt
    Wg = wpe * math.cos(k * wl.h / 2)
    w_leap = 2 / wl.dt * math.asin(Wg * wl.dt / 2)
    assert abs(w_meas / w_leap - 1) < 2e-3, (w_meas, w_leap)
    # the uncorrected plasma frequency differs by the (kh)^2 grid term only
    assert abs(w_meas / wpe - 1) < (k * wl.h) ** 2
    kin, fld = np.array(kin), np.array(fld)
    # total energy at integer steps: field energy plus the mean of the two
    # neighbouring half-step kinetic energies
    e = fld[1:] + 0.5 * (kin[1:] + kin[:-1])
    # the momentum-conserving CIC scheme does not conserve energy exactly: a few
    # per cent oscillation at w dt = 0.2, but no secular drift
    assert (e.max() - e.min()) / e.mean() < 0.08
    per = int(round(2 * math.pi / (w_meas * wl.dt)))
    assert abs(e[:2 * per].mean() / e[-2 * per:].mean() - 1) < 5e-3
