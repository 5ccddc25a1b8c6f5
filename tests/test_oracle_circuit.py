"""Pins of the oracle's external circuit: the serial RC circuit between the
electrodes (the paragraph describing the simulated system), read as a source
V0 charging the anode through R with the gap capacitance C, the charge the
anode collects in a step flowing onto it once per step after the push. An empty box relaxes towards V0 along the closed
form of that recurrence, and a step whose only event is a known charge landing
on the anode moves the potential by exactly that charge over C."""
import numpy as np

import oracle as O
from tests._cases import bare

E = 1.602176634e-19


def test_empty_box_relaxes_to_source_voltage():
    wl = bare(nx=4, ny=4, nz=16, dt=1e-16, phi_a=0.0)
    R, Cg, V0 = 1.0e3, 1.0e-17, 100.0  # dt / RC = 0.01
    ref = O.Oracle(wl, cg_rtol=1e-13)
    ref.set_circuit(R, Cg, V0)
    a = wl.dt / (R * Cg)
    for n in range(1, 41):
        ref.step(1)
        assert abs(ref.moments()["anode_V"] - V0 * (1.0 - (1.0 - a) ** n)) <= 1e-12 * V0
    # the last solve used the potential before the last update: the vacuum ramp
    v_used = V0 * (1.0 - (1.0 - a) ** 39)
    phi = ref.phi().reshape(wl.nz + 1, wl.ny, wl.nx)
    ramp = v_used * np.arange(wl.nz + 1) / wl.nz
    assert np.abs(phi - ramp[:, None, None]).max() <= 1e-10 * V0


def test_collected_charge_moves_anode_by_q_over_c():
    wl = bare(nx=4, ny=4, nz=16, dt=1e-16, weight=1.0)
    n = 100
    rng = np.random.default_rng(3)
    Lx, Ly, Lz = wl.L
    x = np.column_stack([rng.random(n) * Lx, rng.random(n) * Ly, np.full(n, Lz - 1e-12)])
    v = np.column_stack([np.zeros((n, 2)), np.full(n, 1e6)])
    wl.preload = [(x, v), (np.zeros((0, 3)), np.zeros((0, 3))), (np.zeros((0, 3)), np.zeros((0, 3)))]
    Cg = 1.0e-15
    ref = O.Oracle(wl, cg_rtol=1e-13)
    ref.set_circuit(1.0e3, Cg, 0.0)  # V0 = V = 0: no current through R in the first step
    ref.step(1)
    m = ref.moments()
    assert m["abs_anode"][0] == n
    q = -n * E * 1.0
    assert abs(m["charge_to_anode_last"] - q) <= 1e-12 * abs(q)
    assert abs(m["anode_V"] - q / Cg) <= 1e-12 * abs(q / Cg)


def test_circuit_off_keeps_the_anode():
    wl = bare(nx=4, ny=4, nz=16, dt=1e-16, phi_a=5.0, weight=1.0)
    x = np.array([[1e-9, 1e-9, wl.L[2] - 1e-12]])
    wl.preload = [(x, np.array([[0.0, 0.0, 1e6]])), (np.zeros((0, 3)), np.zeros((0, 3))),
                  (np.zeros((0, 3)), np.zeros((0, 3)))]
    ref = O.Oracle(wl, cg_rtol=1e-13)
    ref.set_circuit(0.0, 1e-15, 100.0)  # R = 0: off
    ref.step(3)
    assert ref.moments()["abs_anode"][0] == 1
    assert ref.moments()["anode_V"] == 5.0
