"""Checkpoint and resume (pic_save / pic_load) on the GPU.

1. A round trip without steps reproduces the state bit for bit in both stores:
   particles (pids, positions, velocities), the potential, the integer moments
   and the anode potential; the energies agree to summation order.
2. An FP64 run resumed from a checkpoint taken after 3 steps continues like the
   uninterrupted run for 3 more steps, with surface sources (their carries),
   ionization, charge exchange and an external circuit on: integer moments
   equal, particles and phi within 1e-9 (the resumed first step deposits from
   scratch, so sums differ in the last bits); the sources inject every few
   steps, so a lost carry would move an injection.
3. A mixed-store run resumed for one step agrees with the uninterrupted run
   within the mixed per-step bounds (|dx| <= 1e-5 h, |dv| <= 1e-5 max|v|).
4. Refusals leave the target unchanged: another grid, more particles than a
   species holds, a truncated file, a missing file.
"""
import math

import numpy as np
import pytest

from paper_2606_05893_gb300 import workloads as W
from tests._cases import bare, cx_xsec
from tests.gpu_compare import by_pid, compare_integer_moments, periodic_dx

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import torch
    assert torch.cuda.is_available()
    import paper_2606_05893_gb300 as p
    p.load_library()
    return p


def workload(seed, n_preload=3000, capacity=1 << 16, mu=None):
    """The 32x32x64 workload with charge exchange; mu: mean injected
    superparticles per source and step (the carries then matter every few
    steps)."""
    wl = W.config_small(seed=seed, n_preload=n_preload, capacity=capacity)
    wl.xsec = list(wl.xsec) + [cx_xsec(1e-17)]
    if mu is not None:
        for q in wl.sources:
            q.flux_m2s = mu * wl.species[q.species].weight / (math.pi * q.radius ** 2 * wl.dt)
    return wl


def test_round_trip_is_exact(pkg, tmp_path):
    for p in (pkg.PIC_FP64, pkg.PIC_MIXED):
        wl = workload(49)
        a = pkg.Simulation(wl, precision=p, cg_rtol=1e-12, cg_maxit=5000)
        a.step(3)
        path = tmp_path / f"rt{p}.ckpt"
        a.save(path)
        b = pkg.Simulation(wl, precision=p, cg_rtol=1e-12, cg_maxit=5000, preload=False)
        b.load(path)
        ma, mb = a.moments(), b.moments()
        compare_integer_moments(mb, ma)
        assert mb["step"] == ma["step"] and mb["n_cx"] == ma["n_cx"] and mb["anode_V"] == ma["anode_V"]
        assert mb["pushed"] == ma["pushed"]
        ke_rel = 1e-12 if p == pkg.PIC_FP64 else 1e-5  # mixed: FP32 runs of 8 in store order
        for sp in range(3):
            assert mb["kinetic"][sp] == pytest.approx(ma["kinetic"][sp], rel=ke_rel)
            xa, va, pa = by_pid(*a.particles(sp))
            xb, vb, pb = by_pid(*b.particles(sp))
            assert np.array_equal(pa, pb) and np.array_equal(xa, xb) and np.array_equal(va, vb)
        assert mb["field_energy"] == pytest.approx(ma["field_energy"], rel=1e-12)
        assert np.array_equal(a.phi(), b.phi())
        a.close()
        b.close()


def test_resumed_fp64_run_continues_like_the_uninterrupted_one(pkg, tmp_path):
    wl = workload(50, n_preload=4000, mu=0.37)  # injections at steps 2 and 5
    a = pkg.Simulation(wl, precision=pkg.PIC_FP64, cg_rtol=1e-13, cg_maxit=5000)
    pkg.pic_set_circuit(a.h, 0, 1.0e3, 1.0e-15, wl.phi_anode + 40.0)
    a.step(3)
    path = tmp_path / "mid.ckpt"
    a.save(path)
    a.step(3)
    b = pkg.Simulation(wl, precision=pkg.PIC_FP64, cg_rtol=1e-13, cg_maxit=5000, preload=False)
    b.load(path)  # the circuit, the sources' carries and the counters come from the file
    b.step(3)
    ma, mb = a.moments(), b.moments()
    compare_integer_moments(mb, ma)
    assert sum(ma["injected"]) > 0 and ma["n_ionization"] + ma["n_cx"] > 0
    assert abs(mb["anode_V"] - ma["anode_V"]) <= 1e-12 * abs(ma["anode_V"])
    L = np.array(wl.L)
    for sp in range(3):
        xa, va, pa = by_pid(*a.particles(sp))
        xb, vb, pb = by_pid(*b.particles(sp))
        assert np.array_equal(pa, pb)
        if pa.size:
            assert (periodic_dx(xb, xa, L) / L.max()).max() <= 1e-9
            assert np.abs(vb - va).max() <= 1e-9 * np.abs(va).max()
    assert np.abs(b.phi() - a.phi()).max() <= 1e-9 * np.abs(a.phi()).max()
    a.close()
    b.close()


def test_resumed_mixed_run_one_step(pkg, tmp_path):
    wl = workload(51)
    a = pkg.Simulation(wl, precision=pkg.PIC_MIXED, cg_rtol=1e-12, cg_maxit=5000)
    a.step(3)
    path = tmp_path / "mx.ckpt"
    a.save(path)
    a.step(1)
    b = pkg.Simulation(wl, precision=pkg.PIC_MIXED, cg_rtol=1e-12, cg_maxit=5000, preload=False)
    b.load(path)
    b.step(1)
    ma, mb = a.moments(), b.moments()
    for x, y in zip(mb["count"], ma["count"]):
        assert abs(x - y) <= 2
    L = np.array(wl.L)
    for sp in range(3):
        xa, va, pa = by_pid(*a.particles(sp))
        xb, vb, pb = by_pid(*b.particles(sp))
        common, ia, ib = np.intersect1d(pa, pb, return_indices=True)
        assert common.size >= min(pa.size, pb.size) - 2
        if common.size:
            assert periodic_dx(xb[ib], xa[ia], L).max() <= 1e-5 * wl.h
            assert np.abs(vb[ib] - va[ia]).max() <= 1e-5 * np.abs(va).max()
    a.close()
    b.close()


def test_refusals_leave_the_target_unchanged(pkg, tmp_path):
    wl = workload(52)
    a = pkg.Simulation(wl, precision=pkg.PIC_FP64, cg_rtol=1e-12, cg_maxit=5000)
    a.step(2)
    path = tmp_path / "src.ckpt"
    a.save(path)
    counts = a.moments()["count"]
    # another grid
    other = pkg.Simulation(bare(nx=8, ny=8, nz=8, seed=wl.seed), precision=pkg.PIC_FP64)
    with pytest.raises(pkg.PicError):
        other.load(path)
    assert other.moments()["count"] == [0, 0, 0]
    # more particles than a species holds (same configuration otherwise)
    small = pkg.Simulation(workload(52, n_preload=300, capacity=512), precision=pkg.PIC_FP64)
    before = small.moments()["count"]
    with pytest.raises(pkg.PicError) as e:
        small.load(path)
    assert e.value.status == pkg.PIC_ECAPACITY
    assert small.moments()["count"] == before
    # truncated and missing files
    data = path.read_bytes()
    cut = tmp_path / "cut.ckpt"
    cut.write_bytes(data[: len(data) // 2])
    with pytest.raises(pkg.PicError):
        a.load(cut)
    with pytest.raises(pkg.PicError):
        a.load(tmp_path / "missing.ckpt")
    assert a.moments()["count"] == counts
    for s in (a, other, small):
        s.close()
