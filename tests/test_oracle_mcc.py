"""Pins of the oracle's Monte Carlo collisions, Eq. (4): P = 1 - exp(-u n sigma(E) dt),
and of the ionization resolve (e + Cu -> 2e + Cu+, the ion keeps the neutral's
identity and velocity; the energy above the threshold is shared between the
primary and the secondary electron).

1. Constant cross-section against a fixed background density: the number of
   events per step is Binomial(N_e, 1 - exp(-n0 sigma v dt)), i.e. the rate is
   n_e n0 sigma v.
2. Elastic scattering keeps |v| and scatters isotropically.
3. Ionization: E_primary + E_secondary = E - threshold, the primary keeps its
   direction, counts obey 1 e + 1 Cu -> 2 e + 1 Cu+, each victim lies in the
   primary's cell and is used once, and events beyond the cell's neutrals are
   suppressed.
4. The Lotz table lookup reproduces the closed form at the table points and is
   zero at and below threshold.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2606_05893_gb300 import workloads as W
from tests._cases import bare, const_xsec, ionization_cells_case, isotropic, speed_of_eV


def _beam_case(n, E_eV, xsec, seed=11):
    wl = bare(nx=8, ny=8, nz=8, h=1e-8, dt=1e-16, weight=1e-30, xsec=xsec, seed=seed)
    rng = np.random.default_rng(seed)
    L = np.array(wl.L)
    x = (0.25 + 0.5 * rng.random((n, 3))) * L
    v = isotropic(rng, n, speed_of_eV(E_eV))
    wl.preload = [(x, v), (np.zeros((0, 3)), np.zeros((0, 3))), (np.zeros((0, 3)), np.zeros((0, 3)))]
    return wl, x, v


@pytest.mark.parametrize("sigma", [1e-19, 3e-20])
def test_constant_sigma_rate_against_background(sigma):
    n, E = 100_000, 50.0
    u = speed_of_eV(E)
    n0 = 0.02 / (u * sigma * 1e-16)  # P close to 0.02
    wl, x, v = _beam_case(n, E, [const_xsec(W.XS_ELASTIC, sigma)])
    o = O.Oracle(wl, background_density=n0)
    steps = 5
    o.step(steps)
    P = -math.expm1(-u * n0 * sigma * wl.dt)
    N = n * steps
    m = o.moments()
    sd = math.sqrt(N * P * (1 - P))
    assert abs(m["n_elastic"] - N * P) < 5 * sd, (m["n_elastic"], N * P)
    assert m["n_ionization"] == 0


def test_two_channel_split_follows_sigma_ratio():
    n, E = 100_000, 50.0
    u = speed_of_eV(E)
    s_ion, s_el = 2e-20, 6e-20
    n0 = 0.05 / (u * (s_ion + s_el) * 1e-16)
    wl, x, v = _beam_case(n, E, [const_xsec(W.XS_IONIZATION, s_ion, threshold=7.73),
                                 const_xsec(W.XS_ELASTIC, s_el)])
    o = O.Oracle(wl, background_density=n0)
    o.step(4)
    m = o.moments()
    P = -math.expm1(-u * n0 * (s_ion + s_el) * wl.dt)
    N = 4 * n
    tot = m["n_ionization"] + m["n_elastic"]
    assert abs(tot - N * P) < 5 * math.sqrt(N * P * (1 - P))
    f = s_ion / (s_ion + s_el)
    assert abs(m["n_ionization"] - tot * f) < 5 * math.sqrt(tot * f * (1 - f))


def test_elastic_keeps_speed_and_is_isotropic():
    n, E = 50_000, 20.0
    u = speed_of_eV(E)
    wl, x, v = _beam_case(n, E, [const_xsec(W.XS_ELASTIC, 1e-19)])
    # all electrons initially along +x: scattered ones must lose the x preference
    v[:] = [u, 0.0, 0.0]
    wl.preload[0] = (x, v)
    n0 = 0.5 / (u * 1e-19 * 1e-16)
    o = O.Oracle(wl, background_density=n0)
    o.step()
    xs, vs, pid = o.particles(0)
    speed = np.linalg.norm(vs, axis=1)
    assert np.allclose(speed, u, rtol=1e-14)
    scattered = np.abs(vs[:, 0] - u) > 1e-6 * u
    k = scattered.sum()
    assert k > 0.3 * n
    dirs = vs[scattered] / u
    for c in range(3):
        assert abs(dirs[:, c].mean()) < 5 / math.sqrt(3 * k)
        assert abs((dirs[:, c] ** 2).mean() - 1 / 3) < 5 * math.sqrt(4 / 45 / k)


def test_ionization_energy_split_counts_and_victims():
    wl = ionization_cells_case()
    o = O.Oracle(wl, cg_rtol=1e-13)
    (xe0, ve0), (xn0, vn0), (xi0, vi0) = wl.preload
    ne0, nn0, ni0 = xe0.shape[0], xn0.shape[0], xi0.shape[0]
    o.step()
    m = o.moments()
    log = o.ionization_log()
    nion = m["n_ionization"]
    assert nion == log.shape[0] and nion > 50
    assert m["n_suppressed"] >= 10
    assert m["abs_cathode"] == [0, 0, 0] and m["abs_anode"] == [0, 0, 0]
    assert m["count"] == [ne0 + nion, nn0 - nion, ni0 + nion]
    # pids: electrons 0..ne0-1, neutrals ne0.., ions after; secondaries from next_pid on
    E0 = 100.0
    xe, ve, pe = o.particles(0)
    xn, vn, pn = o.particles(1)
    xi, vi, pi = o.particles(2)
    be = {int(p): k for k, p in enumerate(pe)}
    bi = {int(p): k for k, p in enumerate(pi)}
    h = wl.h
    victims = set()
    for prim, vic, sec in log:
        a, b = ve[be[int(prim)]], ve[be[int(sec)]]
        E1 = 0.5 * W.M_E * a @ a / W.E_CHARGE
        E2 = 0.5 * W.M_E * b @ b / W.E_CHARGE
        assert abs(E1 + E2 - (E0 - W.CU_IONIZATION_EV)) < 1e-12 * E0
        v0 = ve0[int(prim)]
        cross = np.cross(a, v0)
        assert np.linalg.norm(cross) <= 1e-12 * np.linalg.norm(a) * np.linalg.norm(v0)
        assert a @ v0 > 0
        # the victim became an ion with its own velocity, in the primary's cell
        k = int(vic) - ne0
        assert 0 <= k < nn0 and int(vic) not in victims
        victims.add(int(vic))
        assert np.array_equal(vi[bi[int(vic)]], vn0[k])
        assert np.array_equal(np.floor(xn0[k] / h), np.floor(xe0[int(prim)] / h))
        # secondary starts at the primary's new position
        assert np.array_equal(xe[be[int(sec)]], xe[be[int(prim)]])
    # secondaries got consecutive pids in increasing primary-pid order
    assert np.all(np.diff(log[:, 0].astype(np.int64)) > 0)
    first = ne0 + nn0 + ni0
    assert np.array_equal(log[:, 2], np.arange(first, first + nion, dtype=np.uint32))
    # the two-neutral cell converted exactly its two neutrals
    sparse_vic = [v for v in victims if v - ne0 >= 400]
    assert len(sparse_vic) == 2


def test_lotz_table_lookup():
    wl = W.config_tiny()
    o = O.Oracle(wl, preload=False)
    E, s = W.lotz_table(256)
    assert o.sigma(0, W.CU_IONIZATION_EV) == 0.0
    assert o.sigma(0, 5.0) == 0.0
    for i in (1, 17, 100, 255):
        assert o.sigma(0, E[i]) == pytest.approx(s[i], rel=1e-15)
    # closed form between points, within the table's linear-interpolation error
    a = 4.5e-18
    for e in (10.0, 21.0, 100.0, 3000.0):
        exact = a * math.log(e / 7.73) / (e * 7.73)
        assert o.sigma(0, e) == pytest.approx(exact, rel=2e-3)
    assert o.sigma(0, 2e5) == s[-1]
    assert o.sigma(1, 1e-3) == W.ELASTIC_SIGMA_M2


def test_ionization_secondary_direction_isotropic():
    """The secondary electron of an ionization leaves isotropically (reading of
    the ionization kinematics under Eq. 4): cos(theta) uniform on [-1, 1] and the
    azimuth uniform on (-pi, pi], whatever the primary's direction. Checked on
    about two thousand events of one step by the first two moments of cos(theta)
    against 1/3 and 0 (3 standard errors), Kolmogorov-Smirnov tests of cos(theta)
    and of the azimuth, and no correlation with the primary's direction."""
    from scipy import stats
    wl = ionization_cells_case(seed=9, n_dense_e=6000, n_dense_n=8000)
    o = O.Oracle(wl, cg_rtol=1e-13)
    o.step()
    log = o.ionization_log()
    n = log.shape[0]
    assert n > 1500
    xe, ve, pe = o.particles(0)
    be = {int(p): k for k, p in enumerate(pe)}
    sec = np.array([ve[be[int(s)]] for s in log[:, 2]])
    prim = np.array([ve[be[int(p)]] for p in log[:, 0]])
    speed = np.linalg.norm(sec, axis=1)
    keep = speed > 0
    u = sec[keep] / speed[keep, None]
    ct = u[:, 2]
    m = ct.size
    assert abs(ct.mean()) <= 3.0 * math.sqrt(1.0 / 3.0 / m)
    assert abs((ct ** 2).mean() - 1.0 / 3.0) <= 3.0 * math.sqrt(4.0 / 45.0 / m)
    assert stats.kstest(ct, "uniform", args=(-1.0, 2.0)).pvalue > 1e-3
    az = np.arctan2(u[:, 1], u[:, 0])
    assert stats.kstest(az, "uniform", args=(-math.pi, 2.0 * math.pi)).pvalue > 1e-3
    for c in range(3):
        assert abs(u[:, c].mean()) <= 3.0 * math.sqrt(1.0 / 3.0 / m)
    pu = prim[keep] / np.linalg.norm(prim[keep], axis=1)[:, None]
    cos_between = np.einsum("ij,ij->i", u, pu)
    assert abs(cos_between.mean()) <= 3.0 * math.sqrt(1.0 / 3.0 / m)
