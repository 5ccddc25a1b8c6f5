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
