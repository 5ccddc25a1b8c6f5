"""Several instances in one handle step concurrently, each on its own stream:
every instance must give what it gives alone (integers exactly, floats to the
FP64 parity tolerance), and the sort interval (set at run time, as the
autotuner does) reorders particles without changing results."""
import numpy as np
import pytest

from paper_2606_05893_gb300 import workloads as W
from tests.gpu_compare import by_pid, compare_integer_moments

pytestmark = pytest.mark.gpu

TOL = 1e-9


@pytest.fixture(scope="module")
def pkg():
    import torch
    assert torch.cuda.is_available()
    import paper_2606_05893_gb300 as p
    p.load_library()
    return p


def same_particles(sa, ia, sb, ib, L):
    for sp in range(3):
        xa, va, pa = by_pid(*sa.particles(sp, ia))
        xb, vb, pb = by_pid(*sb.particles(sp, ib))
        assert np.array_equal(pa, pb)
        if pa.size:
            d = np.abs(xa - xb)
            d[:, :2] = np.minimum(d[:, :2], np.array(L[:2]) - d[:, :2])
            assert d.max() <= TOL * max(L)
            assert np.abs(va - vb).max() <= TOL * np.abs(vb).max()


def test_instances_in_one_handle_match_separate_handles(pkg):
    wa = W.config_small(seed=3, n_preload=3000)
    wb = W.config_tiny(seed=4, n_preload=800)
    both = pkg.Simulation([wa, wb], cg_rtol=1e-13, cg_maxit=5000)
    a = pkg.Simulation(wa, cg_rtol=1e-13, cg_maxit=5000)
    b = pkg.Simulation(wb, cg_rtol=1e-13, cg_maxit=5000)
    for _ in range(3):
        both.step(2)
        a.step(2)
        b.step(2)
    compare_integer_moments(both.moments(0), a.moments())
    compare_integer_moments(both.moments(1), b.moments())
    same_particles(both, 0, a, 0, wa.L)
    same_particles(both, 1, b, 0, wb.L)
    for s in (both, a, b):
        s.close()


def test_sort_interval_changes_order_only(pkg):
    wl = W.config_small(seed=6, n_preload=5000)
    s1 = pkg.Simulation(wl, cg_rtol=1e-13, cg_maxit=5000)
    s2 = pkg.Simulation(wl, cg_rtol=1e-13, cg_maxit=5000)
    pkg.pic_set_sort_interval(s1.h, 0, 3)
    pkg.pic_set_sort_interval(s2.h, 0, 0)
    s1.step(7)
    s2.step(7)
    compare_integer_moments(s1.moments(), s2.moments())
    same_particles(s1, 0, s2, 0, wl.L)
    with pytest.raises(pkg.PicError):
        pkg.pic_set_sort_interval(s1.h, 0, -1)
    s1.close()
    s2.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_ensemble_steps_are_one_recorded_launch(pkg, precision):
    """Steps in which every instance qualifies for recording run as one graph
    launch for the whole handle (each instance a branch) and give what the
    instances give alone; a sort step of one instance falls back to stepping
    the instances one by one."""
    prec = pkg.PIC_FP64 if precision == "fp64" else pkg.PIC_MIXED
    wls = [W.config_small(seed=31, n_preload=2500), W.config_tiny(seed=32, n_preload=700),
           W.config_small(seed=33, n_preload=1500)]
    for w in wls:
        w.sort_interval = 6
    both = pkg.Simulation(wls, precision=prec, cg_rtol=1e-13, cg_maxit=5000)
    alone = [pkg.Simulation(w, precision=prec, cg_rtol=1e-13, cg_maxit=5000) for w in wls]
    both.step(2)  # step 0 deposits from scratch and sorts; step 1 is recorded
    for s in alone:
        s.step(2)
    l0 = pkg.pic_launch_count()
    both.step(3)  # steps 2-4: replays of two parity patterns, one launch each
    assert pkg.pic_launch_count() - l0 == 3
    both.step(5)  # steps 5-9: step 6 sorts every instance (stepped one by one)
    for s in alone:
        s.step(8)
    for i, w in enumerate(wls):
        compare_integer_moments(both.moments(i), alone[i].moments())
        if precision == "fp64":
            same_particles(both, i, alone[i], 0, w.L)
        else:
            for sp in range(3):
                xa, va, pa = by_pid(*both.particles(sp, i))
                xb, vb, pb = by_pid(*alone[i].particles(sp, 0))
                assert np.array_equal(pa, pb)
                if pa.size:
                    d = np.abs(xa - xb)
                    d[:, :2] = np.minimum(d[:, :2], np.array(w.L[:2]) - d[:, :2])
                    assert d.max() <= 1e-5 * max(w.L)
    for s in [both] + alone:
        s.close()
