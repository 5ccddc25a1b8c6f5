"""Pins of the oracle against the numbers the paper prints for its runs
(tests/golden/paper_setup_parameters.txt, the paragraph that sets up the
simulations, after Eq. 4): the three (F_ext, V0) pairs with a grounded cathode
fix one gap h_gap = V0 / F_ext; in that gap the vacuum solve of Eq. (1) must give
the printed field everywhere, an electron at rest must pick up e F_ext dt_PIC / m_e
towards the anode in one push, and the printed circuit (R = 1 kOhm, C = 1 pF)
must leave the anode effectively constant over one heat step, as the paper
states: one collected electron moves it by e / C and the source restores it with
the recurrence's closed form."""
import math
import os

import numpy as np
import pytest

import oracle as O
from paper_2606_05893_gb300 import workloads as W
from tests._cases import bare

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_setup_parameters.txt")


def _load():
    rows = {}
    with open(GOLDEN) as f:
        for line in f:
            line = line.split("#", 1)[0].split()
            if not line:
                continue
            key, vals = line[0], []
            for t in line[1:]:
                try:
                    vals.append(float(t))
                except ValueError:
                    break  # the units column
            rows.setdefault(key, []).append(vals)
    return rows


P = _load()
FIELDS = [tuple(r) for r in P["field"]]
NZ = 16


def _gap():
    return FIELDS[0][1] / FIELDS[0][0]


def test_printed_field_cases_share_one_gap():
    gaps = [V0 / F for F, V0 in FIELDS]
    assert len(gaps) == 3
    assert max(gaps) - min(gaps) <= 1e-15 * max(gaps)
    assert abs(gaps[0] - 436.8e-9) <= 1e-12 * 436.8e-9


@pytest.mark.parametrize("F_ext,V0", FIELDS)
def test_vacuum_field_is_the_printed_external_field(F_ext, V0):
    h = _gap() / NZ
    wl = bare(nx=4, ny=4, nz=NZ, h=h, dt=P["dt_pic"][0][0], phi_c=0.0, phi_a=V0, weight=P["weight_sp"][0][0])
    ref = O.Oracle(wl, cg_rtol=1e-14)
    ref.step(1)
    rng = np.random.default_rng(7)
    pts = rng.random((200, 3)) * np.array(wl.L)
    E = ref.gather(pts)
    # E = -grad(phi): the anode is positive, so the field points to the cathode
    assert np.abs(E[:, :2]).max() <= 1e-10 * F_ext
    assert np.abs(E[:, 2] + F_ext).max() <= 1e-10 * F_ext
    phi = ref.phi().reshape(NZ + 1, 4, 4)
    z = np.arange(NZ + 1) * h
    assert np.abs(phi - (F_ext * z)[:, None, None]).max() <= 1e-11 * V0


@pytest.mark.parametrize("F_ext,V0", FIELDS)
def test_electron_from_rest_accelerates_to_the_anode(F_ext, V0):
    # one superparticle of the printed weight on the centre node: its own field
    # vanishes there by symmetry (periodic x/y, the two electrodes equidistant)
    h = _gap() / NZ
    dt = P["dt_pic"][0][0]
    wl = bare(nx=4, ny=4, nz=NZ, h=h, dt=dt, phi_c=0.0, phi_a=V0, weight=P["weight_sp"][0][0])
    x0 = np.array([[2 * h, 2 * h, (NZ // 2) * h]])
    empty = (np.zeros((0, 3)), np.zeros((0, 3)))
    wl.preload = [(x0, np.zeros((1, 3))), empty, empty]
    ref = O.Oracle(wl, cg_rtol=1e-14)
    ref.step(1)
    x, v, _ = ref.particles(0)
    dv = W.E_CHARGE * F_ext * dt / W.M_E  # 7.9e3 .. 9.7e3 m/s
    assert v[0, 2] > 0.0
    assert abs(v[0, 2] - dv) <= 1e-9 * dv
    assert np.abs(v[0, :2]).max() <= 1e-9 * dv
    assert abs(x[0, 2] - (x0[0, 2] + dv * dt)) <= 1e-9 * dv * dt


def test_printed_circuit_keeps_the_anode_effectively_constant():
    F_ext, V0 = FIELDS[1]
    R, Cg = P["circuit_R"][0][0], P["circuit_C"][0][0]
    dt = P["dt_pic"][0][0]
    steps = round(P["dt_heat"][0][0] / dt)  # PIC steps in one heat step
    assert steps == 200
    h = _gap() / NZ
    wl = bare(nx=4, ny=4, nz=NZ, h=h, dt=dt, phi_c=0.0, phi_a=V0, weight=P["weight_sp"][0][0])
    x0 = np.array([[1.5 * h, 1.5 * h, wl.L[2] - 1e-12]])
    empty = (np.zeros((0, 3)), np.zeros((0, 3)))
    wl.preload = [(x0, np.array([[0.0, 0.0, 1e6]])), empty, empty]
    ref = O.Oracle(wl, cg_rtol=1e-13)
    ref.set_circuit(R, Cg, V0)
    ref.step(1)
    m = ref.moments()
    assert m["abs_anode"][0] == 1
    jump = -W.E_CHARGE / Cg  # one electron of weight 1 onto 1 pF: -0.16 uV
    assert abs((m["anode_V"] - V0) - jump) <= 1e-6 * abs(jump)
    ref.step(steps - 1)
    a = dt / (R * Cg)
    expect = jump * (1.0 - a) ** (steps - 1)
    dev = ref.moments()["anode_V"] - V0
    # FP64 rounding of V ~ 2e2 V over 200 updates is ~1e-11 V: 1e-4 of the jump
    assert abs(dev - expect) <= 1e-4 * abs(jump)
    assert abs(dev) <= 1e-9 * V0
    assert math.isclose(a * (steps - 1), 1.99e-5, rel_tol=1e-12)
