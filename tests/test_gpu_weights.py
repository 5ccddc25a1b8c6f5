"""Variable-weight particles (integer multiplicities) on the GPU against the oracle.

FP64 path: the particles matched by pid (with their multiplicities, bit-exact),
the event counts, the ionization log, the next pid (3 per successful event) and
the per-cell neutral counts are exact; positions, velocities, rho and phi agree
within 1e-10 after one step (1e-9 over several); the weighted moments (kinetic
energy, total charge, absorbed energy and charge) agree within 1e-10 relative.
Cases: ionization between unequal multiplicities (partial conversions of
victims, secondaries of the moved part, the primary's energy loss drawn with
probability ms / mp), charge exchange together with ionization, a plasma run
with field, injection, absorption and sorting, and unit multiplicities. Mixed
path: the same integer outcomes and multiplicities on the exchange case.
A weighted checkpoint resumes like the uninterrupted run. Also the uploads and
the checkpoint loads that the library refuses.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2606_05893_gb300 import workloads as W
from tests._cases import cx_cells_case, ionization_cells_case, weighted_ionization_case, with_multiplicities
from tests.gpu_compare import compare_integer_moments
from tests.test_gpu_parity import RTOL_SOLVE, full_compare, run_pair

pytestmark = pytest.mark.gpu

FLOAT_KEYS = ("kinetic", "abs_energy_cathode", "abs_energy_anode")


@pytest.fixture(scope="module")
def pkg():
    import torch
    assert torch.cuda.is_available()
    import paper_2606_05893_gb300 as p
    p.load_library()
    return p


def _mult_by_pid(obj, sp):
    pid = obj.particles(sp)[2]
    m = obj.multiplicity(sp)
    o = np.argsort(pid, kind="stable")
    return pid[o], m[o]


def compare_weighted(sim, ref, wl, tol=1e-10):
    mg, mo = full_compare(sim, ref, wl, tol=tol)
    for sp in range(len(wl.species)):
        pg, mgw = _mult_by_pid(sim, sp)
        po, mow = _mult_by_pid(ref, sp)
        assert np.array_equal(pg, po)
        assert np.array_equal(mgw, mow), f"species {sp}: multiplicities differ"
    for k in FLOAT_KEYS:
        for a, b in zip(mg[k], mo[k]):
            assert math.isclose(a, b, rel_tol=tol, abs_tol=1e-40), (k, a, b)
    qscale = max(abs(s.charge_C * s.weight) for s in wl.species)
    assert abs(mg["total_charge"] - mo["total_charge"]) <= tol * max(abs(mo["total_charge"]), qscale)
    for k in ("charge_to_cathode_last", "charge_to_anode_last"):
        assert abs(mg[k] - mo[k]) <= tol * max(abs(mo[k]), qscale), (k, mg[k], mo[k])
    return mg, mo


def test_weighted_ionization_one_step(pkg):
    wl = weighted_ionization_case(seed=8)
    sim, ref = run_pair(pkg, wl, 1)
    mg, _ = compare_weighted(sim, ref, wl)
    assert mg["n_ionization"] > 20 and mg["n_suppressed"] > 0
    assert np.array_equal(sim.ionization_log(), ref.ionization_log())
    # some victims were converted only in part: preloaded neutrals (pids ne ..
    # ne + nn - 1, after the ne electrons) live on with a lower multiplicity
    ne, m_init = wl.preload[0][0].shape[0], wl.preload[1][2]
    pn, mn = _mult_by_pid(sim, 1)
    orig = (pn >= ne) & (pn < ne + m_init.size)
    assert np.any(mn[orig] < m_init[pn[orig] - ne])


def test_weighted_ionization_several_steps_with_sorting(pkg):
    wl = weighted_ionization_case(seed=10)
    wl.sort_interval = 2  # the sort carries multiplicities and meets partial tombstones
    sim, ref = run_pair(pkg, wl, 4)
    compare_weighted(sim, ref, wl, tol=1e-9)
    assert np.array_equal(sim.ionization_log(), ref.ionization_log())


def test_weighted_primary_energy_loss(pkg):
    # primaries of multiplicity 4, victims of 1: a quarter of the primaries lose energy
    wl = weighted_ionization_case(seed=9, m_e=(4, 4), m_n=(1, 1), n_dense_e=1500, n_dense_n=4000)
    sim, ref = run_pair(pkg, wl, 1)
    mg, _ = compare_weighted(sim, ref, wl)
    assert mg["n_ionization"] > 200


def test_weighted_exchange_and_ionization(pkg):
    wl = with_multiplicities(cx_cells_case(seed=23, sigma_ion=1e-10, with_electrons=True), 1, 5, seed=12)
    sim, ref = run_pair(pkg, wl, 2)
    mg, _ = compare_weighted(sim, ref, wl, tol=1e-9)
    assert mg["n_cx"] > 20 and mg["n_ionization"] > 10
    assert np.array_equal(sim.ionization_log(), ref.ionization_log())


def test_weighted_plasma_run(pkg):
    # field, injection (multiplicity 1), absorption at both electrodes, sorting
    wl = with_multiplicities(W.config_tiny(seed=5), 1, 6, seed=3)
    wl.sort_interval = 3
    sim, ref = run_pair(pkg, wl, 10)
    mg, _ = compare_weighted(sim, ref, wl, tol=1e-9)
    assert sum(mg["injected"]) > 0 and sum(mg["abs_anode"]) > 0


def test_unit_multiplicities(pkg):
    wl = ionization_cells_case(seed=4)
    wl.variable_weights = True
    wl.preload = [(x, v, np.ones(x.shape[0], dtype=np.uint32)) for x, v in wl.preload]
    sim, ref = run_pair(pkg, wl, 2)
    mg, _ = compare_weighted(sim, ref, wl, tol=1e-9)
    n0 = sum(p[0].shape[0] for p in wl.preload)
    assert mg["next_pid"] == n0 + 3 * (mg["n_ionization"] + mg["n_cx"])


def test_weighted_mixed_store(pkg):
    # every decision here has P = 1 (exchange and ionization) or comes from
    # Philox alone (victims, the primary's energy loss)
    wl = with_multiplicities(cx_cells_case(seed=25, sigma_ion=1e-10, with_electrons=True), 1, 5, seed=13)
    sim = pkg.Simulation(wl, precision=pkg.PIC_MIXED, cg_rtol=1e-12, cg_maxit=5000)
    ref = O.Oracle(wl, cg_rtol=1e-12)
    sim.step()
    ref.step()
    compare_integer_moments(sim.moments(), ref.moments())
    for sp in range(3):
        pg, mgw = _mult_by_pid(sim, sp)
        po, mow = _mult_by_pid(ref, sp)
        assert np.array_equal(pg, po) and np.array_equal(mgw, mow)
    sim.close()
    ref.close()


def test_weighted_checkpoint_resumes(pkg, tmp_path):
    wl = weighted_ionization_case(seed=10)
    wl.sort_interval = 2
    a = pkg.Simulation(wl, cg_rtol=RTOL_SOLVE, cg_maxit=5000)
    a.step(2)
    path = str(tmp_path / "w.ckpt")
    a.save(path)
    b = pkg.Simulation(weighted_ionization_case(seed=10), cg_rtol=RTOL_SOLVE, cg_maxit=5000, preload=False)
    b.load(path)
    for sp in range(3):  # the round trip is exact, multiplicities included
        pa, ma = _mult_by_pid(a, sp)
        pb, mb = _mult_by_pid(b, sp)
        assert np.array_equal(pa, pb) and np.array_equal(ma, mb)
    a.step(2)
    b.step(2)
    compare_integer_moments(b.moments(), a.moments())
    for sp in range(3):
        xa, va, pa = a.particles(sp)
        xb, vb, pb = b.particles(sp)
        oa, ob = np.argsort(pa), np.argsort(pb)
        assert np.array_equal(pa[oa], pb[ob])
        assert np.array_equal(_mult_by_pid(a, sp)[1], _mult_by_pid(b, sp)[1])
        assert np.abs(xa[oa] - xb[ob]).max(initial=0.0) <= 1e-9 * max(wl.L)
        assert np.abs(va[oa] - vb[ob]).max(initial=0.0) <= 1e-9 * np.abs(va).max(initial=1.0)
    # a weighted checkpoint does not load into an instance without variable weights
    plain = pkg.Simulation(ionization_cells_case(seed=10), cg_rtol=RTOL_SOLVE, cg_maxit=5000, preload=False)
    with pytest.raises(pkg.PicError):
        plain.load(path)
    a.close()
    b.close()
    plain.close()


def test_refusals(pkg):
    wl = weighted_ionization_case(seed=8)
    sim = pkg.Simulation(wl, cg_rtol=RTOL_SOLVE, cg_maxit=5000)
    x = np.full((1, 3), 1e-8)
    v = np.zeros((1, 3))
    with pytest.raises(pkg.PicError):
        pkg.pic_inject_particles_m(sim.h, 0, 0, x, v, np.zeros(1, dtype=np.uint32))
    with pytest.raises(pkg.PicError):  # above 2^24 (the FP32 deposit's exact range)
        pkg.pic_inject_particles_m(sim.h, 0, 0, x, v, np.full(1, (1 << 24) + 1, dtype=np.uint32))
    sim.close()
    plain = pkg.Simulation(ionization_cells_case(seed=4), cg_rtol=RTOL_SOLVE, cg_maxit=5000)
    with pytest.raises(pkg.PicError):
        pkg.pic_inject_particles_m(plain.h, 0, 0, x, v, np.full(1, 2, dtype=np.uint32))
    pkg.pic_inject_particles_m(plain.h, 0, 0, x, v, np.ones(1, dtype=np.uint32))
    assert np.all(plain.multiplicity(0) == 1)
    plain.close()


def test_weighted_and_plain_instances_in_one_handle(pkg):
    # per-instance flags: a weighted and a plain instance step together (the
    # handle's ensemble step) and each matches its own oracle run
    from tests.gpu_compare import compare_particles
    wls = [weighted_ionization_case(seed=8), ionization_cells_case(seed=3)]
    sim = pkg.Simulation(wls, precision=pkg.PIC_FP64, cg_rtol=RTOL_SOLVE, cg_maxit=5000)
    refs = [O.Oracle(w, cg_rtol=RTOL_SOLVE) for w in wls]
    for _ in range(2):
        sim.step()
        for r in refs:
            r.step()
    for i, (w, r) in enumerate(zip(wls, refs)):
        compare_integer_moments(sim.moments(i), r.moments())
        for sp in range(3):
            compare_particles(sim, r, w, sp, 1e-9, 1e-9, inst=i)
            pg = sim.particles(sp, inst=i)[2]
            mg = sim.multiplicity(sp, inst=i)
            po, mo = _mult_by_pid(r, sp)
            o = np.argsort(pg, kind="stable")
            assert np.array_equal(pg[o], po) and np.array_equal(mg[o], mo)
        r.close()
    sim.close()
