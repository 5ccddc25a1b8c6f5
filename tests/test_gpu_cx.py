"""Charge exchange (resonant Cu+ + Cu) on the GPU against the oracle.

FP64 path: the exchanges, suppressions and ionizations, the ionization log and
the per-cell neutral counts are bit-exact, particles, rho and phi agree within
1e-10 after one step (1e-9 over several), including steps that sort the stores
with the exchanged ions' tombstones in them and a step with more events than
the single-block event ordering takes. Mixed path: the same integer outcomes
(every decision here has P = 1 or a wide margin) and the per-step bounds of the
mixed tests. Also the rate against a fixed background at the ion's energy, an
exchange channel inside a plasma run with field, injection and sorting, and the
configurations the library refuses.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2606_05893_gb300 import workloads as W
from tests._cases import bare, cx_cells_case, cx_xsec, isotropic
from tests.gpu_compare import compare_integer_moments
from tests.test_gpu_mixed import check_step
from tests.test_gpu_parity import full_compare, run_pair

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import torch
    assert torch.cuda.is_available()
    import paper_2606_05893_gb300 as p
    p.load_library()
    return p


def test_exchange_cells_one_step(pkg):
    wl = cx_cells_case()
    sim, ref = run_pair(pkg, wl, 1)
    mg, _ = full_compare(sim, ref, wl)
    assert mg["n_cx"] == 67 and mg["n_suppressed"] == 63


def test_exchange_cells_several_steps_with_sorting(pkg):
    wl = cx_cells_case(seed=22)
    wl.sort_interval = 2  # sorts meet the tombstones of exchanged ions and neutrals
    sim = pkg.Simulation(wl, precision=pkg.PIC_FP64, cg_rtol=1e-13, cg_maxit=5000)
    ref = O.Oracle(wl, cg_rtol=1e-13)
    for _ in range(5):
        sim.step()
        ref.step()
        compare_integer_moments(sim.moments(), ref.moments())
    mg, _ = full_compare(sim, ref, wl, tol=1e-9)
    assert mg["n_cx"] >= 5 * 67


def test_exchange_and_ionization_share_victims(pkg):
    wl = cx_cells_case(seed=23, sigma_ion=1e-10, with_electrons=True)
    sim, ref = run_pair(pkg, wl, 2)
    mg, _ = full_compare(sim, ref, wl, tol=1e-9)
    assert mg["n_cx"] > 0 and mg["n_ionization"] > 0 and mg["n_suppressed"] > 0
    assert np.array_equal(sim.ionization_log(), ref.ionization_log())


def test_exchange_many_events(pkg):
    # more events than the single-block event ordering takes (2048)
    wl = cx_cells_case(seed=24, sigma_ion=1e-10, with_electrons=True, n_dense_i=2600, n_dense_n=2300)
    sim, ref = run_pair(pkg, wl, 1)
    mg, _ = full_compare(sim, ref, wl)
    assert mg["n_cx"] + mg["n_ionization"] + mg["n_suppressed"] > 2048 and mg["n_suppressed"] > 0
    assert np.array_equal(sim.ionization_log(), ref.ionization_log())


def test_exchange_mixed_store(pkg):
    wl = cx_cells_case(seed=25, sigma_ion=1e-10, with_electrons=True)
    sim = pkg.Simulation(wl, precision=pkg.PIC_MIXED, cg_rtol=1e-12, cg_maxit=5000)
    ref = O.Oracle(wl, cg_rtol=1e-12)
    sim.step()
    ref.step()
    compare_integer_moments(sim.moments(), ref.moments())
    check_step(sim, ref, wl, allow_count=0)
    assert sim.moments()["n_cx"] > 0
    for _ in range(2):  # recorded steps replayed
        sim.step()
        ref.step()
    compare_integer_moments(sim.moments(), ref.moments())


def test_background_rate_at_the_ion_energy_bit_exact(pkg):
    n, E_i, dt = 20000, 50.0, 1e-14
    u = math.sqrt(2.0 * E_i * W.E_CHARGE / W.M_CU)
    sigma = 1e-19 + (E_i - 1.0) / 99.0 * (1e-17 - 1e-19)
    n0 = 0.3 / (u * sigma * dt)
    wl = bare(nx=8, ny=8, nz=8, h=1e-8, dt=dt, weight=1e-30, capacity=1 << 16, seed=9,
              xsec=[cx_xsec([1e-19, 1e-17], E=[1.0, 100.0])])
    rng = np.random.default_rng(9)
    x = (0.25 + 0.5 * rng.random((n, 3))) * np.array(wl.L)
    empty = (np.zeros((0, 3)), np.zeros((0, 3)))
    wl.preload = [empty, empty, (x, isotropic(rng, n, u))]
    sim, ref = run_pair(pkg, wl, 3, background_density=n0)
    mg, mo = sim.moments(), ref.moments()
    assert mg["n_cx"] == mo["n_cx"]
    P = -math.expm1(-0.3)
    assert abs(mg["n_cx"] - 3 * n * P) < 5 * math.sqrt(3 * n * P)


def test_exchange_in_plasma_run(pkg):
    wl = W.config_small(seed=44, n_preload=4000)
    wl.xsec = list(wl.xsec) + [cx_xsec(1e-17)]
    sim, ref = run_pair(pkg, wl, 6)
    mg, _ = full_compare(sim, ref, wl, tol=1e-9)
    assert mg["n_cx"] > 0


@pytest.mark.parametrize("bad", ["electron_projectile", "product_not_target", "weights", "other_target"])
def test_refused_configurations(pkg, bad):
    wl = cx_cells_case(sigma_ion=1e-10, with_electrons=True)
    X = wl.xsec[0]
    if bad == "electron_projectile":
        wl.xsec[0] = W.XSec(X.kind, 0, X.target, X.product, X.threshold_eV, X.E_eV, X.sigma_m2)
    elif bad == "product_not_target":
        wl.xsec[0] = W.XSec(X.kind, X.projectile, X.target, 2, X.threshold_eV, X.E_eV, X.sigma_m2)
    elif bad == "weights":
        wl.species[2] = W.Species(*[getattr(wl.species[2], f) for f in ("name", "charge_C", "mass_kg")], 2.0,
                                  wl.species[2].role, wl.species[2].capacity)
        wl.xsec = wl.xsec[:1]
    else:
        # a second neutral species as the exchange's target, the ionization keeping species 1
        wl.species.append(W.Species("Cu2", 0.0, W.M_CU, wl.species[1].weight, W.NEUTRAL, 1024))
        wl.preload.append((np.zeros((0, 3)), np.zeros((0, 3))))
        wl.xsec[0] = W.XSec(X.kind, X.projectile, 3, 3, X.threshold_eV, X.E_eV, X.sigma_m2)
    with pytest.raises(pkg.PicError):
        pkg.Simulation(wl, precision=pkg.PIC_FP64)
