"""Surface-coupling output on the GPU: the ions absorbed at the cathode (pid,
species, crossing step, the point where the path meets z = 0, v^{n+1/2},
energy) against the oracle's log of the same run. The runs step through
recorded graphs after their first steps, so the log is also checked inside
replays."""
import numpy as np
import pytest

import oracle as O
from tests._cases import cathode_hits_case

pytestmark = pytest.mark.gpu

E_CHARGE = 1.602176634e-19


@pytest.fixture(scope="module")
def pkg():
    import torch
    assert torch.cuda.is_available()
    import paper_2606_05893_gb300 as p
    p.load_library()
    return p


def run_pair(pkg, wl, steps, precision, cap=4096):
    sim = pkg.Simulation(wl, precision=precision, cg_rtol=1e-13)
    pkg.pic_set_hit_log(sim.h, 0, cap)
    ref = O.Oracle(wl, cg_rtol=1e-13)
    sim.step(steps)
    ref.step(steps)
    return sim, ref


def check_against(g, o, wl, tol_x, tol_v):
    assert np.array_equal(g["pid"], o["pid"])
    assert np.array_equal(g["step"], o["step"].astype(np.int64))
    assert np.array_equal(g["species"], o["species"])
    assert g["lost"] == 0
    assert np.all(g["x"][:, 2] == 0.0)
    # periodic distance: a crossing on the x = Lx face may land at either end
    d = np.abs(g["x"][:, :2] - o["xy"])
    L = np.array(wl.L[:2])
    assert np.minimum(d, L - d).max() <= tol_x
    vmax = np.abs(o["v"]).max()
    assert np.abs(g["v"] - o["v"]).max() <= tol_v * vmax
    m = wl.species[2].mass_kg
    ke = 0.5 * m * (o["v"] ** 2).sum(1) / E_CHARGE
    assert np.abs(g["ke_eV"] - ke).max() <= 2 * tol_v * ke.max() + 1e-300


def test_hits_fp64_match_oracle(pkg):
    wl, k = cathode_hits_case()
    sim, ref = run_pair(pkg, wl, 10, pkg.PIC_FP64)
    g, o = pkg.pic_get_hits(sim.h, 0), ref.hits()
    assert g["pid"].size == np.count_nonzero(k < 10) > 0
    check_against(g, o, wl, 1e-10 * max(wl.L), 1e-12)
    # the read emptied the log; the rest arrive later
    assert pkg.pic_get_hits(sim.h, 0)["pid"].size == 0
    sim.step(4)
    ref.step(4)
    check_against(pkg.pic_get_hits(sim.h, 0), ref.hits(), wl, 1e-10 * max(wl.L), 1e-12)
    sim.close()


def test_hits_mixed_store(pkg):
    # FP32 offsets and velocities: the crossing point carries their rounding
    wl, k = cathode_hits_case(seed=13)
    sim, ref = run_pair(pkg, wl, 12, pkg.PIC_MIXED)
    check_against(pkg.pic_get_hits(sim.h, 0), ref.hits(), wl, 1e-5 * wl.h, 1e-6)
    sim.close()


def test_hits_in_applied_field(pkg):
    # the vacuum field of a positive anode speeds the ions towards the cathode
    wl, k = cathode_hits_case(seed=14)
    wl.phi_anode = 1.0e3
    sim, ref = run_pair(pkg, wl, 12, pkg.PIC_FP64)
    check_against(pkg.pic_get_hits(sim.h, 0), ref.hits(), wl, 1e-10 * max(wl.L), 1e-10)
    sim.close()


def test_hit_log_overflow_and_off(pkg):
    wl, k = cathode_hits_case(seed=15)
    sim, ref = run_pair(pkg, wl, 6, pkg.PIC_FP64, cap=5)
    o = ref.hits()
    assert o["pid"].size > 5
    # room for fewer hits than are waiting: refused, nothing copied, log kept
    with pytest.raises(pkg.PicError):
        pkg.pic_get_hits(sim.h, 0, cap=2)
    g = pkg.pic_get_hits(sim.h, 0, cap=5)
    assert g["pid"].size == 5 and g["lost"] == o["pid"].size - 5
    # which five are kept is not specified; each is a real hit with its step
    where = {int(p_): i for i, p_ in enumerate(o["pid"])}
    assert all(int(p_) in where for p_ in g["pid"])
    assert all(g["step"][i] == o["step"][where[int(p_)]] for i, p_ in enumerate(g["pid"]))
    assert pkg.pic_get_hits(sim.h, 0)["lost"] == 0
    pkg.pic_set_hit_log(sim.h, 0, 0)
    with pytest.raises(pkg.PicError):
        pkg.pic_get_hits(sim.h, 0)
    sim.close()
