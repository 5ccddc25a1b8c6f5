"""Moments (a11) on the GPU: kinetic energy per species, field energy and total
charge against the oracle and against a host recomputation from what the
library hands back (particles, phi).

Against the oracle the bounds follow from the per-step state tolerances, with
eps_v = 1e-10 (FP64) or 1e-5 (mixed) of max|v| per velocity and eps_phi = 1e-10
or 1e-7 of the potential scale per node: |dKE| <= (m w / 2) sum(2 |v| dv + dv^2)
with dv = eps_v max|v|, and |dW| <= (eps0 h / 2) sum over edges (2 |d| e + e^2)
with e = 2 eps_phi scale, both evaluated on the oracle's state. Against the
host recomputation: FP64 within 1e-12 (only the summation differs); mixed KE
within 1e-5 (squares in FP32, the velocities' own precision); mixed field
energy, formed from the solver's FP32 hi/lo state, within the rounding of its
FP32 edge differences, |dd| <= 4 u (|d| + |dvac|) per edge (u = 2^-24, dvac the
vacuum step of a z edge), plus 27 u of the sum for the FP32 squares and runs.
"""
import numpy as np
import pytest

import oracle as O
from paper_2606_05893_gb300 import workloads as W
from tests._cases import cx_cells_case

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import torch
    assert torch.cuda.is_available()
    import paper_2606_05893_gb300 as p
    p.load_library()
    return p


def host_field_energy(phi, wl):
    f = phi.reshape(wl.nz + 1, wl.ny, wl.nx)
    dx = np.roll(f, -1, axis=2) - f
    dy = np.roll(f, -1, axis=1) - f
    dz = f[1:] - f[:-1]
    return 0.5 * W.EPS0 * wl.h * (np.sum(dx * dx) + np.sum(dy * dy) + np.sum(dz * dz))


def mixed_fe_rounding_bound(phi, wl):
    u = 2.0 ** -24
    f = phi.reshape(wl.nz + 1, wl.ny, wl.nx)
    dvac = abs(wl.phi_anode - wl.phi_cathode) / wl.nz
    dxy = np.concatenate([(np.roll(f, -1, axis=2) - f).ravel(), (np.roll(f, -1, axis=1) - f).ravel()])
    dz = (f[1:] - f[:-1]).ravel()
    e_xy = 4 * u * np.abs(dxy)
    e_z = 4 * u * (np.abs(dz) + dvac)
    rounding = np.sum(2 * np.abs(dxy) * e_xy + e_xy ** 2) + np.sum(2 * np.abs(dz) * e_z + e_z ** 2)
    total = np.sum(dxy ** 2) + np.sum(dz ** 2)
    return 0.5 * W.EPS0 * wl.h * float(rounding + 27 * u * total)


def host_kinetic(sim, wl, sp):
    _, v, _ = sim.particles(sp)
    s = wl.species[sp]
    return 0.5 * s.mass_kg * s.weight * float(np.sum(v.astype(np.float64) ** 2))


CASES = {
    "small": lambda: W.config_small(seed=46, n_preload=6000),
    "exchange": lambda: cx_cells_case(seed=26, sigma_ion=1e-10, with_electrons=True),
}


def ke_bound(ref, wl, sp, eps_v):
    _, v, _ = ref.particles(sp)
    if v.shape[0] == 0:
        return 0.0
    sp_ = wl.species[sp]
    speed = np.linalg.norm(v, axis=1)
    dv = eps_v * np.abs(v).max() * np.sqrt(3.0)
    return 0.5 * sp_.mass_kg * sp_.weight * float(np.sum(2.0 * speed * dv + dv * dv))


def fe_bound(ref, wl, eps_phi):
    phi = ref.phi()
    qw = max(abs(s.charge_C * s.weight) for s in wl.species)
    cells = [np.floor(x / wl.h).astype(np.int64) for (x, _), s in zip(wl.preload, wl.species) if s.charge_C != 0]
    cells = np.concatenate(cells)
    npc = np.unique(cells, axis=0, return_counts=True)[1].max() if len(cells) else 1
    e = 2.0 * eps_phi * max(np.abs(phi).max(), npc * qw / (W.EPS0 * wl.h))
    f = phi.reshape(wl.nz + 1, wl.ny, wl.nx)
    d = np.concatenate([(np.roll(f, -1, axis=2) - f).ravel(), (np.roll(f, -1, axis=1) - f).ravel(),
                        (f[1:] - f[:-1]).ravel()])
    return 0.5 * W.EPS0 * wl.h * float(np.sum(2.0 * np.abs(d) * e + e * e))


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_moments_match_oracle_and_host(pkg, case, precision):
    wl = CASES[case]()
    p = pkg.PIC_FP64 if precision == "fp64" else pkg.PIC_MIXED
    rtol = 1e-13 if precision == "fp64" else 1e-12
    sim = pkg.Simulation(wl, precision=p, cg_rtol=rtol, cg_maxit=5000)
    ref = O.Oracle(wl, cg_rtol=rtol)
    sim.step()
    ref.step()
    mg, mo = sim.moments(), ref.moments()
    eps_v, eps_phi = (1e-10, 1e-10) if precision == "fp64" else (1e-5, 1e-7)
    host_ke_tol = 1e-12 if precision == "fp64" else 1e-5
    for sp in range(len(wl.species)):
        ko, kg = mo["kinetic"][sp], mg["kinetic"][sp]
        assert abs(kg - ko) <= ke_bound(ref, wl, sp, eps_v), (sp, kg, ko)
        kh = host_kinetic(sim, wl, sp)
        assert abs(kg - kh) <= host_ke_tol * kh, (sp, kg, kh)
    fo, fg = mo["field_energy"], mg["field_energy"]
    assert fo > 0 and abs(fg - fo) <= fe_bound(ref, wl, eps_phi), (fg, fo)
    phi_g = sim.phi()
    fh = host_field_energy(phi_g, wl)
    host_fe_tol = 1e-12 * fh if precision == "fp64" else mixed_fe_rounding_bound(phi_g, wl)
    assert abs(fg - fh) <= host_fe_tol, (fg, fh)
    assert mg["total_charge"] == pytest.approx(mo["total_charge"], rel=1e-14, abs=1e-30)
    sim.close()


def test_field_energy_of_the_vacuum_gap(pkg):
    # an empty box: E = -V/L_z everywhere, so the energy is eps0 V^2 L_x L_y / (2 L_z)
    # on the node grid (the edge sum is exact for a linear potential); the mixed
    # store forms the edge differences and squares in FP32 (27 u of the sum)
    from tests._cases import bare
    wl = bare(nx=32, ny=16, nz=48, h=5e-9, phi_a=250.0)
    for p in (pkg.PIC_FP64, pkg.PIC_MIXED):
        sim = pkg.Simulation(wl, precision=p, cg_rtol=1e-12)
        sim.step()
        Lx, Ly, Lz = wl.L
        exact = 0.5 * W.EPS0 * 250.0 ** 2 * Lx * Ly / Lz
        tol = 1e-9 if p == pkg.PIC_FP64 else 27 * 2.0 ** -24
        assert abs(sim.moments()["field_energy"] - exact) <= tol * exact
        sim.close()
