"""External RC circuit on the GPU (pic_set_circuit) against the oracle: the
anode potential step by step, the potential and the particles of a plasma run
with the circuit on, the relaxation of an empty box in both stores, and a
circuit switched on between recorded steps."""
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


def test_plasma_run_with_circuit_matches_oracle(pkg):
    wl = W.config_small(seed=41, n_preload=4000)
    R, Cg, V0 = 1.0e3, 1.0e-15, wl.phi_anode + 50.0
    sim = pkg.Simulation(wl, cg_rtol=1e-13, cg_maxit=5000)
    ref = O.Oracle(wl, cg_rtol=1e-13)
    pkg.pic_set_circuit(sim.h, 0, R, Cg, V0)
    ref.set_circuit(R, Cg, V0)
    moved = 0.0
    for _ in range(8):
        sim.step(1)
        ref.step(1)
        mg, mo = sim.moments(), ref.moments()
        compare_integer_moments(mg, mo)
        assert abs(mg["anode_V"] - mo["anode_V"]) <= 1e-12 * abs(mo["anode_V"])
        moved = max(moved, abs(mo["anode_V"] - wl.phi_anode))
    assert moved > 1e-3  # the circuit did move the anode
    assert np.abs(sim.phi() - ref.phi()).max() <= 1e-9 * np.abs(ref.phi()).max()
    for sp in range(3):
        compare_particles(sim, ref, wl, sp, 1e-9, 1e-9)
    sim.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_empty_box_relaxes(pkg, precision):
    p = pkg.PIC_FP64 if precision == "fp64" else pkg.PIC_MIXED
    wl = bare(nx=4, ny=4, nz=16, dt=1e-16, phi_a=0.0)
    R, Cg, V0 = 1.0e3, 1.0e-17, 100.0
    sim = pkg.Simulation(wl, precision=p, cg_rtol=1e-12)
    pkg.pic_set_circuit(sim.h, 0, R, Cg, V0)
    a = wl.dt / (R * Cg)
    for n in range(1, 21):
        sim.step(1)
        assert abs(sim.moments()["anode_V"] - V0 * (1.0 - (1.0 - a) ** n)) <= 1e-12 * V0
    # the last solve used the potential before the last update: the vacuum ramp
    # (the mixed store solves relative to the configured anode voltage and
    # carries the circuit's offset in FP32: its rounding, ~6e-8 of the offset)
    v_used = V0 * (1.0 - (1.0 - a) ** 19)
    phi = sim.phi().reshape(wl.nz + 1, wl.ny, wl.nx)
    ramp = v_used * np.arange(wl.nz + 1) / wl.nz
    tol = 1e-9 if precision == "fp64" else 1e-7
    assert np.abs(phi - ramp[:, None, None]).max() <= tol * V0
    sim.close()


def test_circuit_switched_on_between_recorded_steps(pkg):
    wl = W.config_small(seed=42, n_preload=3000)
    sim = pkg.Simulation(wl, cg_rtol=1e-13, cg_maxit=5000)
    ref = O.Oracle(wl, cg_rtol=1e-13)
    sim.step(4)  # steps recorded and replayed without a circuit
    ref.step(4)
    assert sim.moments()["anode_V"] == wl.phi_anode
    R, Cg, V0 = 1.0e3, 1.0e-15, wl.phi_anode - 30.0
    pkg.pic_set_circuit(sim.h, 0, R, Cg, V0)
    ref.set_circuit(R, Cg, V0)
    sim.step(4)
    ref.step(4)
    mg, mo = sim.moments(), ref.moments()
    assert mo["anode_V"] != wl.phi_anode
    assert abs(mg["anode_V"] - mo["anode_V"]) <= 1e-12 * abs(mo["anode_V"])
    compare_integer_moments(mg, mo)
    pkg.pic_set_circuit(sim.h, 0, 0.0, 0.0, 0.0)  # off: the anode stays where it is
    v = sim.moments()["anode_V"]
    sim.step(2)
    assert sim.moments()["anode_V"] == v
    sim.close()


def test_two_instances_keep_their_own_circuit_and_hit_log(pkg):
    # one handle, two instances stepping concurrently on their own streams:
    # instance 0 with a circuit and a hit log, instance 1 with neither
    from tests._cases import cathode_hits_case
    wa = W.config_small(seed=43, n_preload=3000)
    wb, _ = cathode_hits_case(seed=16)
    wb.phi_anode = 500.0
    sim = pkg.Simulation([wa, wb], cg_rtol=1e-13, cg_maxit=5000)
    ra, rb = O.Oracle(wa, cg_rtol=1e-13), O.Oracle(wb, cg_rtol=1e-13)
    R, Cg, V0 = 1.0e3, 1.0e-15, wa.phi_anode + 20.0
    pkg.pic_set_circuit(sim.h, 0, R, Cg, V0)
    ra.set_circuit(R, Cg, V0)
    pkg.pic_set_hit_log(sim.h, 1, 1024)
    for _ in range(6):
        sim.step(1)
        ra.step(1)
        rb.step(1)
    ma, mb = sim.moments(0), sim.moments(1)
    assert abs(ma["anode_V"] - ra.moments()["anode_V"]) <= 1e-12 * abs(ra.moments()["anode_V"])
    assert mb["anode_V"] == wb.phi_anode
    compare_integer_moments(ma, ra.moments())
    compare_integer_moments(mb, rb.moments())
    g, o = pkg.pic_get_hits(sim.h, 1), rb.hits()
    assert g["pid"].size > 0 and np.array_equal(g["pid"], o["pid"])
    with pytest.raises(pkg.PicError):
        pkg.pic_get_hits(sim.h, 0)  # instance 0 has no log
    sim.close()
