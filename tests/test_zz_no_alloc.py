"""The Poisson solve that allocates nothing, for callers that cannot allocate
device memory while they run: its work vectors live in a fixed array inside the
library. Calls go through the C ABI on caller-owned device buffers and must
reproduce both the handle-based pic_solve and the CPU oracle's solve within
the 1e-10 relative tolerance of the other FP64 parity tests (all solved to a
1e-13 residual, or 1e-12 where a degenerate grid converges in a handful of
iterations), on two calls in a row; the device's free memory must not move
across a call; sizes beyond the fixed array are refused with a clear error.

This file is collected last on purpose (test_zz_*): a failure here leaves
every other test already run.
"""
import numpy as np
import pytest

from tests._cases import bare

pytestmark = pytest.mark.gpu

RTOL = 1e-13
TOL = 1e-10


def _solve_static(pkg, torch, wl, rho, phi0=None, rtol=RTOL, maxit=100000):
    nx, ny, nz = wl.nx, wl.ny, wl.nz
    rho_dev = torch.from_numpy(np.ascontiguousarray(rho)).cuda()
    if phi0 is None:
        phi_dev = torch.zeros((nz + 1, ny, nx), dtype=torch.float64, device="cuda")
    else:
        phi_dev = torch.from_numpy(np.ascontiguousarray(phi0)).cuda()
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream().cuda_stream
    st, iters, rel = pkg.pic_poisson_solve_static(nx, ny, nz, wl.h, wl.phi_cathode, wl.phi_anode,
                                                  rho_dev.data_ptr(), phi_dev.data_ptr(), rtol, maxit, stream)
    return st, iters, rel, phi_dev.cpu().numpy()


def test_static_solve_matches_pic_solve_and_oracle_twice():
    import torch
    assert torch.cuda.is_available()
    import oracle
    import paper_2606_05893_gb300 as pkg
    pkg.load_library()
    nx, ny, nz = 24, 20, 34
    wl = bare(nx=nx, ny=ny, nz=nz, h=2.5e-9, phi_c=-2.0, phi_a=400.0)
    rng = np.random.default_rng(17)
    sim = pkg.Simulation(wl, cg_rtol=RTOL, cg_maxit=20000, preload=False)
    for call in range(2):
        rho = rng.standard_normal((nz + 1, ny, nx)) * 2e6 * (call + 1)
        ref, _, rel_ref = sim.solve(rho)
        assert rel_ref <= RTOL
        orc = oracle.poisson(nx, ny, nz, wl.h, wl.phi_cathode, wl.phi_anode, rho, rtol=RTOL)[0]
        st, iters, rel, phi = _solve_static(pkg, torch, wl, rho)
        assert st == pkg.PIC_OK, pkg.pic_last_error(None)
        assert rel <= RTOL and iters > 0
        assert np.abs(phi - ref).max() <= TOL * np.abs(ref).max()
        assert np.abs(phi - orc).max() <= TOL * np.abs(orc).max()
    sim.close()


def test_static_solve_allocates_no_device_memory():
    import torch
    import oracle
    import paper_2606_05893_gb300 as pkg
    pkg.load_library()
    nx, ny, nz = 16, 16, 40
    wl = bare(nx=nx, ny=ny, nz=nz, h=2.5e-9, phi_c=0.0, phi_a=50.0)
    rho = np.random.default_rng(3).standard_normal((nz + 1, ny, nx)) * 1e6
    orc = oracle.poisson(nx, ny, nz, wl.h, wl.phi_cathode, wl.phi_anode, rho, rtol=RTOL)[0]
    stream = torch.cuda.current_stream().cuda_stream
    rho_dev = torch.from_numpy(rho).cuda()
    phi_dev = torch.zeros((nz + 1, ny, nx), dtype=torch.float64, device="cuda")
    # first call: the library's kernels and its fixed array may be loaded on first use
    st, _, _ = pkg.pic_poisson_solve_static(nx, ny, nz, wl.h, wl.phi_cathode, wl.phi_anode, rho_dev.data_ptr(),
                                            phi_dev.data_ptr(), RTOL, 100000, stream)
    assert st == pkg.PIC_OK, pkg.pic_last_error(None)
    phi_dev.zero_()
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    st, iters, rel = pkg.pic_poisson_solve_static(nx, ny, nz, wl.h, wl.phi_cathode, wl.phi_anode,
                                                  rho_dev.data_ptr(), phi_dev.data_ptr(), RTOL, 100000, stream)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert st == pkg.PIC_OK and iters > 0
    assert free1 == free0, f"free device memory moved by {free0 - free1} bytes across the call"
    phi = phi_dev.cpu().numpy()
    assert np.abs(phi - orc).max() <= TOL * np.abs(orc).max()


@pytest.mark.parametrize("shape", [(8, 6, 2), (12, 1, 10), (1, 1, 9)])
def test_static_solve_degenerate_grids(shape):
    """nz = 2 (one unknown plane takes both electrode terms), ny = 1 and nx = ny = 1."""
    import torch
    import oracle
    import paper_2606_05893_gb300 as pkg
    pkg.load_library()
    nx, ny, nz = shape
    wl = bare(nx=nx, ny=ny, nz=nz, h=2.5e-9, phi_c=1.5, phi_a=-30.0)
    rho = np.random.default_rng(nx * 100 + nz).standard_normal((nz + 1, ny, nx)) * 3e6
    orc = oracle.poisson(nx, ny, nz, wl.h, wl.phi_cathode, wl.phi_anode, rho, rtol=1e-12)[0]
    st, iters, rel, phi = _solve_static(pkg, torch, wl, rho, rtol=1e-12)
    assert st == pkg.PIC_OK, pkg.pic_last_error(None)
    assert rel <= 1e-12
    assert np.abs(phi - orc).max() <= TOL * np.abs(orc).max()


def test_static_solve_initial_guess_limit_and_zero_problem():
    import torch
    import oracle
    import paper_2606_05893_gb300 as pkg
    pkg.load_library()
    nx, ny, nz = 10, 12, 16
    wl = bare(nx=nx, ny=ny, nz=nz, h=2.5e-9, phi_c=0.0, phi_a=20.0)
    rng = np.random.default_rng(5)
    rho = rng.standard_normal((nz + 1, ny, nx)) * 2e6
    orc = oracle.poisson(nx, ny, nz, wl.h, wl.phi_cathode, wl.phi_anode, rho, rtol=RTOL)[0]
    # a nonzero initial guess near the solution converges to the same potential
    guess = orc + rng.standard_normal(orc.shape) * 1e-3 * np.abs(orc).max()
    st, it_guess, rel, phi = _solve_static(pkg, torch, wl, rho, phi0=guess)
    assert st == pkg.PIC_OK, pkg.pic_last_error(None)
    assert np.abs(phi - orc).max() <= TOL * np.abs(orc).max()
    # one iteration cannot reach 1e-13: PIC_ENOCONV with the iteration count and a message
    st, iters, rel, _ = _solve_static(pkg, torch, wl, rho, maxit=1)
    assert st == pkg.PIC_ENOCONV and iters == 1 and rel > RTOL
    assert "residual" in pkg.pic_last_error(None)
    # rho = 0 between grounded electrodes: the zero solution, no iteration
    wl0 = bare(nx=nx, ny=ny, nz=nz, h=2.5e-9, phi_c=0.0, phi_a=0.0)
    st, iters, rel, phi = _solve_static(pkg, torch, wl0, np.zeros_like(rho), phi0=guess)
    assert st == pkg.PIC_OK and iters == 0 and rel == 0.0
    assert not phi.any()


def test_static_solve_rejects_oversize_grid():
    import torch
    import paper_2606_05893_gb300 as pkg
    pkg.load_library()
    stream = torch.cuda.current_stream().cuda_stream
    nx, ny, nz = 64, 64, 66  # 64*64*65 unknowns > PIC_STATIC_MAX_UNKNOWNS
    assert nx * ny * (nz - 1) > pkg.PIC_STATIC_MAX_UNKNOWNS
    dummy = torch.zeros(8, dtype=torch.float64, device="cuda")
    st, _, _ = pkg.pic_poisson_solve_static(nx, ny, nz, 1e-9, 0.0, 1.0, dummy.data_ptr(), dummy.data_ptr(), 1e-8,
                                            100, stream)
    assert st == pkg.PIC_EINVAL
    assert "PIC_STATIC_MAX_UNKNOWNS" in pkg.pic_last_error(None)
