"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle.

FP64 path, one step from an identical state: integer outputs (counts per
species, injected/absorbed/ionization/elastic/suppressed counts, pids, sort
permutations, neutral cell counts, the ionization log) are bit-exact; floats
agree within 1e-10 relative (positions / L, velocities / max|v|, rho and phi in
the max norm), with both Poisson solves run to a 1e-13 relative residual so
that the solver tolerance does not mask the comparison.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2606_05893_gb300 import workloads as W
from tests._cases import bare, const_xsec, ionization_cells_case, isotropic, speed_of_eV
from tests.gpu_compare import compare_integer_moments, compare_particles, rel_inf

pytestmark = pytest.mark.gpu

TOL = 1e-10
RTOL_SOLVE = 1e-13


@pytest.fixture(scope="module")
def pkg():
    import torch
    assert torch.cuda.is_available()
    import paper_2606_05893_gb300 as p
    p.load_library()
    return p


def run_pair(pkg, wl, steps, precision=0, **kw):
    sim = pkg.Simulation(wl, precision=precision, cg_rtol=RTOL_SOLVE, cg_maxit=5000, **kw)
    ref = O.Oracle(wl, cg_rtol=RTOL_SOLVE, **({"background_density": kw["background_density"]}
                                               if "background_density" in kw else {}))
    for _ in range(steps):
        sim.step()
        ref.step()
    return sim, ref


def full_compare(sim, ref, wl, tol=TOL):
    mg, mo = sim.moments(), ref.moments()
    compare_integer_moments(mg, mo)
    for sp in range(len(wl.species)):
        compare_particles(sim, ref, wl, sp, tol, tol)
    # max-norm comparison, floored at one superparticle's charge density and
    # potential scale (the grids can cancel to rounding noise, e.g. when
    # electrons and ions sit on the same spot)
    qw = max(abs(s.charge_C * s.weight) for s in wl.species)
    rho_g, rho_o = sim.rho(), ref.rho()
    assert np.abs(rho_g - rho_o).max() <= tol * max(np.abs(rho_o).max(), qw / wl.h ** 3)
    phi_g, phi_o = sim.phi(), ref.phi()
    assert np.abs(phi_g - phi_o).max() <= tol * max(np.abs(phi_o).max(), qw / (W.EPS0 * wl.h))
    for sp, s in enumerate(wl.species):
        if s.role == W.NEUTRAL:
            assert np.array_equal(sim.ncount(sp), ref.ncount(sp))
    return mg, mo


def test_device_philox_matches_oracle(pkg):
    sim = pkg.Simulation(W.config_tiny(), preload=False)
    rng = np.random.default_rng(0)
    for _ in range(20):
        ctr = rng.integers(0, 2 ** 32, 4, dtype=np.uint64).astype(np.uint32)
        key = rng.integers(0, 2 ** 32, 2, dtype=np.uint64).astype(np.uint32)
        out = pkg.pic_philox(sim.h, 64, ctr, key)
        for i in (0, 1, 31, 63):
            c = ctr.copy()
            c[0] = np.uint32((int(ctr[0]) + i) & 0xFFFFFFFF)
            assert np.array_equal(out[i], O.philox(c, key))
    sim.close()


@pytest.mark.parametrize("shape", [(16, 16, 32), (8, 8, 16), (6, 10, 12), (5, 7, 9), (32, 32, 64)])
def test_poisson_solve_matches_oracle(pkg, shape):
    nx, ny, nz = shape
    wl = bare(nx=nx, ny=ny, nz=nz, h=2.5e-9, phi_c=-3.0, phi_a=250.0)
    rng = np.random.default_rng(nx * 100 + nz)
    rho = rng.standard_normal((nz + 1, ny, nx)) * 3e6
    sim = pkg.Simulation(wl, cg_rtol=RTOL_SOLVE, cg_maxit=20000, preload=False)
    phi_g, it, rel = sim.solve(rho)
    assert rel <= RTOL_SOLVE
    phi_o, ito, relo = O.poisson(nx, ny, nz, wl.h, wl.phi_cathode, wl.phi_anode, rho, rtol=RTOL_SOLVE)
    assert rel_inf(phi_g, phi_o) <= TOL
    if nx % 2 == 0 and ny % 2 == 0 and nx >= 16:
        # the multigrid preconditioner needs far fewer iterations than plain CG
        assert it < ito / 3, (it, ito)
    sim.close()


# The mixed solver's multigrid stops at the first coarse level of at most 70 000
# unknowns whose sides allow the exact fast-diagonalization solve: 16x16x31
# (32x32x64), 32x16x63 (unequal sides), 24x24x47; 10x10x19 (sides not multiples
# of 4) keeps the deeper levels and the cluster kernel.
@pytest.mark.parametrize("shape", [(32, 32, 64), (64, 32, 128), (48, 48, 96), (20, 20, 40)])
def test_poisson_solve_mixed_precision(pkg, shape):
    nx, ny, nz = shape
    wl = bare(nx=nx, ny=ny, nz=nz, h=2.5e-9, phi_c=0.0, phi_a=600.0)
    rng = np.random.default_rng(4 + nx)
    rho = rng.standard_normal((nz + 1, ny, nx)) * 3e6
    sim = pkg.Simulation(wl, precision=pkg.PIC_MIXED, cg_rtol=1e-12, cg_maxit=20000, preload=False)
    phi_g, it, rel = sim.solve(rho)
    assert rel <= 1e-12
    phi_o, _, _ = O.poisson(nx, ny, nz, wl.h, wl.phi_cathode, wl.phi_anode, rho, rtol=1e-13)
    assert rel_inf(phi_g, phi_o) <= 1e-9
    sim.close()


def test_one_step_tiny(pkg):
    wl = W.config_tiny(seed=3)
    sim, ref = run_pair(pkg, wl, 1)
    full_compare(sim, ref, wl)


def test_ten_steps_tiny_with_sorting_and_injection(pkg):
    wl = W.config_tiny(seed=5)
    sim, ref = run_pair(pkg, wl, 10)
    mg, mo = full_compare(sim, ref, wl, tol=1e-9)
    assert sum(mg["injected"]) > 0 and sum(mg["abs_anode"]) > 0


def test_ionization_and_suppression_step(pkg):
    wl = ionization_cells_case(seed=3)
    sim, ref = run_pair(pkg, wl, 1)
    mg, mo = full_compare(sim, ref, wl)
    assert mg["n_ionization"] > 50 and mg["n_suppressed"] >= 10
    lg, lo = sim.ionization_log(), ref.ionization_log()
    assert np.array_equal(lg, lo)


def test_ionization_several_steps(pkg):
    wl = ionization_cells_case(seed=8)
    sim, ref = run_pair(pkg, wl, 4)
    mg, mo = full_compare(sim, ref, wl, tol=1e-9)
    assert np.array_equal(sim.ionization_log(), ref.ionization_log())


def test_ionization_many_events(pkg):
    # more events in one step than the single-block event ordering takes
    # (2048): the radix passes order them
    wl = ionization_cells_case(seed=5, n_dense_e=3000, n_dense_n=2500)
    sim, ref = run_pair(pkg, wl, 1)
    mg, mo = full_compare(sim, ref, wl)
    assert mg["n_ionization"] + mg["n_suppressed"] > 2048 and mg["n_suppressed"] > 0
    assert np.array_equal(sim.ionization_log(), ref.ionization_log())


def test_small_workload_one_step(pkg):
    wl = W.config_small()
    sim, ref = run_pair(pkg, wl, 1)
    full_compare(sim, ref, wl)


def test_small_workload_five_steps(pkg):
    wl = W.config_small(seed=42)
    sim, ref = run_pair(pkg, wl, 5)
    mg, mo = full_compare(sim, ref, wl, tol=1e-9)
    assert mg["n_ionization"] + mg["n_elastic"] > 0


def test_background_rates_bit_exact(pkg):
    n, E = 20000, 50.0
    u = speed_of_eV(E)
    s_ion, s_el = 2e-20, 6e-20
    n0 = 0.05 / (u * (s_ion + s_el) * 1e-16)
    wl = bare(nx=8, ny=8, nz=8, h=1e-8, dt=1e-16, weight=1e-30, capacity=1 << 16,
              xsec=[const_xsec(W.XS_IONIZATION, s_ion, threshold=7.73), const_xsec(W.XS_ELASTIC, s_el)])
    rng = np.random.default_rng(2)
    x = (0.25 + 0.5 * rng.random((n, 3))) * np.array(wl.L)
    wl.preload = [(x, isotropic(rng, n, u)), (np.zeros((0, 3)), np.zeros((0, 3))), (np.zeros((0, 3)), np.zeros((0, 3)))]
    sim, ref = run_pair(pkg, wl, 3, background_density=n0)
    mg, mo = sim.moments(), ref.moments()
    assert mg["n_elastic"] == mo["n_elastic"] and mg["n_ionization"] == mo["n_ionization"]
    P = -math.expm1(-u * n0 * (s_ion + s_el) * wl.dt)
    assert abs(mg["n_elastic"] + mg["n_ionization"] - 3 * n * P) < 5 * math.sqrt(3 * n * P)
    compare_particles(sim, ref, wl, 0, TOL, TOL)


def _breakpoint_electrons(rng, E_tab, n):
    """Electron energies on the ionization table's points, just around its
    threshold and spread log-uniformly over the table (isotropic directions)."""
    k = n // 4
    E = np.concatenate([
        E_tab[rng.integers(1, E_tab.size - 1, k)],
        W.CU_IONIZATION_EV * (1.0 + rng.integers(-40, 41, k) * 1e-7),
        E_tab[rng.integers(1, E_tab.size - 1, k)] * (1.0 + rng.uniform(-3e-6, 3e-6, k)),
        np.exp(rng.uniform(0.0, math.log(5000.0), n - 3 * k)),
    ])
    speed = np.sqrt(2.0 * E * W.E_CHARGE / W.M_E)
    v = rng.standard_normal((n, 3))
    v *= (speed / np.linalg.norm(v, axis=1))[:, None]
    return v


@pytest.mark.parametrize("P_target", [0.02, 0.4])
def test_background_rates_on_table_breakpoints_bit_exact(pkg, P_target):
    # Eq. (4) with the tabulated Lotz ionization cross-section: the kernels
    # decide most collisions in FP32 and fall back to the FP64 rule near table
    # points, thresholds and the U ~ P boundary; every decision must equal the
    # oracle's FP64 one. The large-P case makes 1 - exp(-x) far from x.
    n = 40000
    rng = np.random.default_rng(31)
    xs = W.cu_plasma_xsec()
    wl = bare(nx=8, ny=8, nz=8, h=1e-8, dt=1e-17, weight=1e-30, capacity=1 << 16, xsec=xs)
    u100 = speed_of_eV(100.0)
    n0 = P_target / (u100 * (float(xs[0].sigma_m2.max()) + float(xs[1].sigma_m2[0])) * wl.dt)
    x = (0.3 + 0.4 * rng.random((n, 3))) * np.array(wl.L)
    wl.preload = [(x, _breakpoint_electrons(rng, xs[0].E_eV, n)), (np.zeros((0, 3)), np.zeros((0, 3))),
                  (np.zeros((0, 3)), np.zeros((0, 3)))]
    sim, ref = run_pair(pkg, wl, 2, background_density=n0)
    mg, mo = sim.moments(), ref.moments()
    assert mg["n_ionization"] > 20 and mg["n_elastic"] > 100
    assert mg["n_elastic"] == mo["n_elastic"] and mg["n_ionization"] == mo["n_ionization"]
    compare_particles(sim, ref, wl, 0, TOL, TOL)


def test_host_upload_between_steps(pkg):
    # particles handed over by the host between steps (the surface-model transfer)
    # join the next step's deposit, which the previous step had already started
    wl = W.config_small(seed=13, n_preload=4000)
    sim, ref = run_pair(pkg, wl, 2)
    rng = np.random.default_rng(5)
    for sp, n in ((0, 300), (1, 200), (2, 100)):
        x = rng.random((n, 3)) * np.array(wl.L) * np.array([1.0, 1.0, 0.5])
        v = rng.standard_normal((n, 3)) * (3e5 if sp == 0 else 800.0)
        pkg.pic_inject_particles(sim.h, 0, sp, x, v)
        ref.load(sp, x, v)
    for _ in range(2):
        sim.step()
        ref.step()
    full_compare(sim, ref, wl, tol=1e-9)


def test_sort_permutation_and_offsets_bit_exact(pkg):
    wl = W.config_tiny(seed=9)
    sim = pkg.Simulation(wl)
    ref = O.Oracle(wl)
    sim.sort_now()
    ref.sort()
    for sp in range(3):
        _, _, pg = sim.particles(sp)
        _, _, po = ref.particles(sp)
        assert np.array_equal(pg, po)
        assert np.array_equal(sim.cell_start(sp), ref.cell_start(sp))
    sim.close()


@pytest.mark.parametrize("n_dense", [300, 5000])
def test_sort_crowded_cells_and_dead_slots(pkg, n_dense):
    # one dense cell (n_dense electrons and as many ions: above 4096 the radix
    # path takes over), 400 neutrals and 200 sparse electrons in buckets sorted
    # block-wide, and, right after a step, the dead slots of converted neutrals
    wl = ionization_cells_case(seed=7, n_dense_e=n_dense, capacity=1 << 17)
    sim = pkg.Simulation(wl)
    ref = O.Oracle(wl)
    for _ in range(2):
        sim.step()
        ref.step()
        assert sim.moments()["n_ionization"] > 0
        sim.sort_now()
        ref.sort()
        for sp in range(3):
            _, _, pg = sim.particles(sp)
            _, _, po = ref.particles(sp)
            assert np.array_equal(pg, po), sp
            assert np.array_equal(sim.cell_start(sp), ref.cell_start(sp)), sp
    sim.close()


def test_sort_order_mixed_store(pkg):
    # the mixed store's cells come from FP32 offsets, so cell boundaries may
    # differ from the oracle's by rounding: check the order itself (pids rising
    # inside every cell range, ranges covering the store) and the pid sets
    wl = ionization_cells_case(seed=8, n_dense_e=600, capacity=1 << 15)
    sim = pkg.Simulation(wl, precision=pkg.PIC_MIXED)
    ref = O.Oracle(wl)
    sim.step(2)
    ref.step(2)
    sim.sort_now()
    for sp in range(3):
        _, _, pg = sim.particles(sp)
        _, _, po = ref.particles(sp)
        cs = sim.cell_start(sp)
        assert cs[0] == 0 and cs[-1] == pg.size and np.all(np.diff(cs) >= 0)
        for a, b in zip(cs[:-1], cs[1:]):
            if b - a > 1:
                assert np.all(np.diff(pg[a:b].astype(np.int64)) > 0)
        assert np.array_equal(np.sort(pg), np.sort(po))
    sim.close()


def test_vacuum_uniform_field_push_exact(pkg):
    wl = bare(nx=4, ny=4, nz=16, h=5e-9, dt=1e-16, phi_c=0.0, phi_a=100.0, weight=1e-30)
    rng = np.random.default_rng(1)
    L = np.array(wl.L)
    n = 64
    x0 = rng.random((n, 3)) * L * np.array([1, 1, 0.3]) + np.array([0, 0, 0.2 * L[2]])
    v0 = rng.standard_normal((n, 3)) * 1e5
    wl.preload = [(x0, v0), (np.zeros((0, 3)), np.zeros((0, 3))), (x0.copy(), -v0)]
    sim, ref = run_pair(pkg, wl, 30)
    for sp in (0, 2):
        compare_particles(sim, ref, wl, sp, 1e-12, 1e-12)
