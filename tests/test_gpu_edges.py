"""Edge cases and failure reporting of the C ABI on the GPU (no fault is ever
provoked on the device: every failure here is detected by argument checks,
bounded device counters or solver status and reported as a status code).

- empty stores, a single unknown plane (nz = 2), odd grid sizes (no red-black
  colouring: the solver falls back to a Jacobi preconditioner) against the
  oracle;
- capacity overflow -> PIC_ECAPACITY with the step's state kept;
- iteration limit -> PIC_ENOCONV, non-fatal, the step still advances;
- invalid configurations and arguments -> PIC_EINVAL, no handle;
- the literal "+3 V" small case: no electron gains the 7.73 eV threshold from
  the applied field alone, so ionization stays at zero when the space charge
  is negligible.
"""
import ctypes as C

import numpy as np
import pytest

import oracle as O
from paper_2606_05893_gb300 import workloads as W
from tests._cases import bare
from tests.gpu_compare import compare_integer_moments, compare_particles

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import torch
    assert torch.cuda.is_available()
    import paper_2606_05893_gb300 as p
    p.load_library()
    return p


def test_empty_stores_step(pkg):
    wl = bare(nx=8, ny=8, nz=8, phi_c=0.0, phi_a=10.0)
    sim = pkg.Simulation(wl, cg_rtol=1e-13, cg_maxit=5000)
    ref = O.Oracle(wl, cg_rtol=1e-13)
    sim.step(3)
    ref.step(3)
    m = sim.moments()
    assert m["count"] == [0, 0, 0] and m["step"] == 3
    assert np.abs(sim.phi() - ref.phi()).max() <= 1e-10 * 10.0
    sim.close()


@pytest.mark.parametrize("shape", [(5, 7, 2), (3, 3, 5), (7, 6, 9), (1, 1, 4)])
def test_odd_and_degenerate_grids_match_oracle(pkg, shape):
    nx, ny, nz = shape
    wl = W.config_tiny(seed=11, nx=nx, ny=ny, nz=nz, n_preload=200)
    for prec, tol in ((pkg.PIC_FP64, 1e-9), (pkg.PIC_MIXED, None)):
        sim = pkg.Simulation(wl, precision=prec, cg_rtol=1e-13, cg_maxit=20000)
        ref = O.Oracle(wl, cg_rtol=1e-13)
        sim.step(2)
        ref.step(2)
        if tol is not None:
            compare_integer_moments(sim.moments(), ref.moments())
            for sp in range(3):
                compare_particles(sim, ref, wl, sp, tol, tol)
        phi_g, phi_o = sim.phi(), ref.phi()
        assert np.abs(phi_g - phi_o).max() <= 1e-6 * max(np.abs(phi_o).max(), 1.0)
        sim.close()


def test_capacity_overflow_reports_ecapacity(pkg):
    wl = W.config_tiny(seed=3, capacity=4096)
    for s in wl.species:
        s.capacity = 400  # electrons preload 360, sources inject ~1.6/step
    x, v = wl.preload[0]
    sim = pkg.Simulation(wl)
    with pytest.raises(pkg.PicError) as ei:
        pkg.pic_inject_particles(sim.h, 0, 0, np.repeat(x[:1], 100, 0), np.repeat(v[:1], 100, 0))
    assert ei.value.status == pkg.PIC_ECAPACITY
    assert sim.count(0) == x.shape[0]  # nothing appended
    # a source flooding the store: the step reports the overflow, the handle stays usable
    pkg.pic_inject(sim.h, 0, 0, wl.L[0] / 2, wl.L[1] / 2, wl.L[0] / 4, 1e33, 5800.0)
    st = sim.step(1, check=False)
    assert st == pkg.PIC_ECAPACITY
    assert sim.count(0) <= 400
    assert "capacity" in pkg.pic_last_error(sim.h)
    sim.close()


def test_iteration_limit_is_nonfatal(pkg):
    wl = W.config_small(n_preload=2000)
    sim = pkg.Simulation(wl, cg_rtol=1e-14, cg_maxit=2)
    st = sim.step(1, check=False)
    assert st == pkg.PIC_ENOCONV
    m = sim.moments()
    assert m["step"] == 1 and m["cg_iters"] <= 3 and m["cg_resid_rel"] > 1e-14
    assert sim.step(1, check=False) == pkg.PIC_ENOCONV  # still usable
    sim.close()


def test_invalid_configurations_rejected(pkg):
    L = pkg.load_library()
    good = W.config_tiny()
    for mutate in (lambda c: setattr(c, "nz", 1), lambda c: setattr(c, "h", 0.0), lambda c: setattr(c, "nspecies", 0),
                   lambda c: setattr(c, "precision", 7), lambda c: setattr(c, "cg_rtol", -1.0)):
        holder = pkg._CfgHolder(good, pkg.PIC_FP64, None, None, pkg.PIC_WARM_PREV, None)
        mutate(holder.cfg)
        h = C.c_void_p()
        st = L.pic_create(C.byref(holder.cfg), 1, None, C.byref(h))
        assert st == pkg.PIC_EINVAL and not h.value
        assert pkg.pic_last_error(None)
    # unequal ionization weights
    bad = W.config_tiny()
    bad.species[1].weight *= 2
    with pytest.raises(pkg.PicError) as ei:
        pkg.Simulation(bad)
    assert ei.value.status == pkg.PIC_EINVAL
    sim = pkg.Simulation(good)
    with pytest.raises(pkg.PicError):
        pkg.pic_inject_particles(sim.h, 0, 0, np.array([[-1.0, 0.0, 0.0]]), np.zeros((1, 3)))  # outside
    with pytest.raises(pkg.PicError):
        pkg.pic_inject(sim.h, 0, 9, 0.0, 0.0, 1e-9, 1.0, 1.0)  # bad species
    with pytest.raises(pkg.PicError):
        pkg.pic_moments(sim.h, 3)  # bad instance
    sim.close()


def test_literal_three_volt_case_has_no_ionization(pkg):
    # weight small enough that the space charge cannot heat electrons to 7.73 eV
    wl = W.config_small(anode_V=3.0, weight=1e-6, n_preload=3000)
    for src in wl.sources:  # keep the injected macroparticles per step as at weight 100
        src.flux_m2s *= 1e-6 / 100.0
    sim = pkg.Simulation(wl)
    sim.step(20)
    m = sim.moments()
    assert m["n_ionization"] == 0 and m["n_suppressed"] == 0
    sim.close()


def test_warm_start_zero_matches_previous_phi(pkg):
    wl = W.config_tiny(seed=2)
    a = pkg.Simulation(wl, cg_rtol=1e-13, warm_start=pkg.PIC_WARM_PREV)
    b = pkg.Simulation(wl, cg_rtol=1e-13, warm_start=pkg.PIC_WARM_ZERO)
    a.step(3)
    b.step(3)
    assert np.abs(a.phi() - b.phi()).max() <= 1e-9 * np.abs(a.phi()).max()
    assert b.moments()["cg_iters"] >= a.moments()["cg_iters"]
    a.close()
    b.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_nonfinite_potential_flags_the_moments(pkg, precision):
    """A potential holding NaN (set through pic_set_phi) makes the field energy
    NaN, and pic_moments flags it (PIC_FLAG_NONFINITE) rather than returning a
    NaN moment silently; a finite potential clears the flag. No step runs on the
    NaN potential: the push derives cell indices from positions and is never fed
    non-finite values (uploads refuse them)."""
    import paper_2606_05893_gb300 as p
    wl = W.config_tiny(seed=21)
    sim = p.Simulation(wl, precision=precision)
    sim.step(1)
    assert not sim.moments()["error_flags"] & 32
    phi = sim.phi()
    bad = phi.copy()
    bad[wl.nz // 2, wl.ny // 2, wl.nx // 2] = np.nan
    sim.set_phi(bad)
    m = sim.moments()
    assert m["error_flags"] & 32 and not np.isfinite(m["field_energy"])
    sim.set_phi(phi)
    assert not sim.moments()["error_flags"] & 32
    sim.close()
