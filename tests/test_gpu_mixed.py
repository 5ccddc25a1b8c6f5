"""Mixed-precision path (int32 cell + FP32 offsets/velocities, FP32 deposit, gather,
multigrid smoothing and scattering angles; the refinement residual and update in
float-float arithmetic (about 48 bits), FP64 reductions, and collision decisions
identical to the FP64 rule) against the FP64 oracle.

Per step from an identical state the bounds are |dx| <= 1e-5 h (FP32 offsets
carry 2^-24 h; a particle crossing up to ~10 cells per step adds the FP32
velocity error times v dt), |dv| <= 1e-5 max|v|, |drho| <= 1e-6 of the larger of
max|rho| and the summed magnitude of the contributions to a node (FP32
accumulation when charges cancel), |dphi| <= 1e-7 of the larger of max|phi| and
the potential scale of that summed charge (the FP32 density error, ~1e-7
relative, carries into the space-charge part of phi, which can exceed the
applied potential). Integer outcomes agree
except where an FP32-rounded position or velocity sits on a decision boundary
(absorption, cell index, collision draw); over many steps the trajectories
decorrelate, so the comparison becomes statistical: ensemble means of particle
counts and kinetic energies lie within 3.5 standard errors of the oracle's.
"""
import math
import os

import numpy as np
import pytest

import oracle as O
from paper_2606_05893_gb300 import workloads as W
from tests._cases import ionization_cells_case
from tests.gpu_compare import by_pid, periodic_dx

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import torch
    assert torch.cuda.is_available()
    import paper_2606_05893_gb300 as p
    p.load_library()
    return p


def one_step(pkg, wl):
    sim = pkg.Simulation(wl, precision=pkg.PIC_MIXED, cg_rtol=1e-12, cg_maxit=5000)
    ref = O.Oracle(wl, cg_rtol=1e-12)
    sim.step()
    ref.step()
    return sim, ref


def check_step(sim, ref, wl, allow_count=2):
    mg, mo = sim.moments(), ref.moments()
    for a, b in zip(mg["count"], mo["count"]):
        assert abs(a - b) <= max(allow_count, 1e-4 * b)
    L = np.array(wl.L)
    for sp in range(3):
        xg, vg, pg = by_pid(*sim.particles(sp))
        xo, vo, po = by_pid(*ref.particles(sp))
        common, ig, io = np.intersect1d(pg, po, return_indices=True)
        assert common.size >= min(pg.size, po.size) - allow_count
        if common.size == 0:
            continue
        dx = periodic_dx(xg[ig], xo[io], L).max()
        assert dx <= 1e-5 * wl.h, (sp, dx / wl.h)
        vmax = np.abs(vo).max()
        dv = np.abs(vg[ig] - vo[io]).max() / vmax
        assert dv <= 1e-5, (sp, dv)
    rho_g, rho_o = sim.rho(), ref.rho()
    qw = max(abs(s.charge_C * s.weight) for s in wl.species)
    # largest number of charged particles in one cell at the start of the step
    cells = [np.floor(x / wl.h).astype(np.int64) for (x, _), s in zip(wl.preload, wl.species) if s.charge_C != 0]
    cells = np.concatenate(cells) if cells else np.zeros((0, 3), np.int64)
    npc = np.unique(cells, axis=0, return_counts=True)[1].max() if len(cells) else 1
    scale = max(np.abs(rho_o).max(), npc * qw / wl.h ** 3)
    assert np.abs(rho_g - rho_o).max() <= 1e-6 * scale
    phi_g, phi_o = sim.phi(), ref.phi()
    assert np.abs(phi_g - phi_o).max() <= 1e-7 * max(np.abs(phi_o).max(), npc * qw / (W.EPS0 * wl.h))


def test_mixed_one_step_tiny(pkg):
    wl = W.config_tiny(seed=4)
    sim, ref = one_step(pkg, wl)
    check_step(sim, ref, wl)


def test_mixed_one_step_small(pkg):
    wl = W.config_small()
    sim, ref = one_step(pkg, wl)
    check_step(sim, ref, wl, allow_count=3)


def test_mixed_one_step_ionization(pkg):
    wl = ionization_cells_case(seed=6)
    sim, ref = one_step(pkg, wl)
    check_step(sim, ref, wl, allow_count=3)


def test_mixed_subcase_64x64x128(pkg):
    """The error subcase of the large mixed run: 64x64x128 cells of 1.25 nm,
    ~7.8e5 particles, one step against the FP64 oracle."""
    wl = W.config_mixed_subcase(seed=0)
    sim, ref = one_step(pkg, wl)
    check_step(sim, ref, wl, allow_count=10)


@pytest.mark.parametrize("precision", [0, 1])
def test_solver_host_loop_matches_graph(pkg, precision):
    # the recorded graph and the host-driven loop run the same kernels with
    # fixed-order reductions: identical input, bit-identical phi
    wl = W.config_tiny(seed=2)
    rng = np.random.default_rng(3)
    rho = rng.standard_normal((wl.nz + 1, wl.ny, wl.nx)) * 1e6
    out = []
    for mode in ("1", "0"):
        os.environ["PIC_SOLVER_GRAPH"] = mode
        try:
            sim = pkg.Simulation(wl, precision=precision, cg_rtol=1e-12, cg_maxit=5000, preload=False)
        finally:
            os.environ.pop("PIC_SOLVER_GRAPH", None)
        out.append(sim.solve(rho))
        sim.close()
    assert np.array_equal(out[0][0], out[1][0])
    assert out[0][1] == out[1][1]


@pytest.mark.parametrize("steps,seeds", [(150, 8)])
def test_mixed_ensemble_moments_within_3_sigma(pkg, steps, seeds):
    """Ensembles over seeds: GPU mixed vs FP64 oracle; counts and kinetic energy per
    species at the end agree within 3.5 standard errors of the difference."""
    g_cnt, o_cnt, g_ke, o_ke = [], [], [], []
    for sd in range(seeds):
        wl = W.config_tiny(seed=100 + sd)
        sim = pkg.Simulation(wl, precision=pkg.PIC_MIXED)
        ref = O.Oracle(wl)
        sim.step(steps)
        ref.step(steps)
        mg, mo = sim.moments(), ref.moments()
        g_cnt.append(mg["count"]); o_cnt.append(mo["count"])
        g_ke.append(mg["kinetic"]); o_ke.append(mo["kinetic"])
        sim.close()
    g_cnt, o_cnt = np.array(g_cnt, float), np.array(o_cnt, float)
    g_ke, o_ke = np.array(g_ke), np.array(o_ke)
    for a, b in ((g_cnt, o_cnt), (g_ke, o_ke)):
        for sp in range(a.shape[1]):
            d = a[:, sp] - b[:, sp]
            se = math.sqrt((a[:, sp].var(ddof=1) + b[:, sp].var(ddof=1)) / seeds)
            scale = max(abs(b[:, sp].mean()), 1e-300)
            assert abs(d.mean()) <= 3.5 * se + 1e-9 * scale, (sp, d.mean(), se)
