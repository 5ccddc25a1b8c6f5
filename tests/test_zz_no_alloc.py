"""The Poisson solve that allocates nothing, for callers that cannot allocate
device memory while they run: its work vectors live in a fixed array inside the
library. Two calls in a row through the C ABI, each on caller-owned device
buffers, must reproduce the handle-based pic_solve within the 1e-10 relative
tolerance of the other FP64 parity tests (both solved to a 1e-13 residual),
and sizes beyond the fixed array are refused with a clear error.

This file is collected last on purpose (test_zz_*): a failure here leaves
every other test already run.
"""
import numpy as np
import pytest

from tests._cases import bare

pytestmark = pytest.mark.gpu

RTOL = 1e-13
TOL = 1e-10


def test_static_solve_matches_pic_solve_twice():
    import torch
    assert torch.cuda.is_available()
    import paper_2606_05893_gb300 as pkg
    pkg.load_library()
    nx, ny, nz = 24, 20, 34
    wl = bare(nx=nx, ny=ny, nz=nz, h=2.5e-9, phi_c=-2.0, phi_a=400.0)
    rng = np.random.default_rng(17)
    sim = pkg.Simulation(wl, cg_rtol=RTOL, cg_maxit=20000, preload=False)
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        rho = rng.standard_normal((nz + 1, ny, nx)) * 2e6 * (call + 1)
        ref, _, rel_ref = sim.solve(rho)
        assert rel_ref <= RTOL
        rho_dev = torch.from_numpy(rho).cuda()
        phi_dev = torch.zeros((nz + 1, ny, nx), dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        st, iters, rel = pkg.pic_poisson_solve_static(nx, ny, nz, wl.h, wl.phi_cathode, wl.phi_anode,
                                                      rho_dev.data_ptr(), phi_dev.data_ptr(), RTOL, 100000, stream)
        assert st == pkg.PIC_OK, pkg.pic_last_error(None)
        assert rel <= RTOL and iters > 0
        phi = phi_dev.cpu().numpy()
        assert np.abs(phi - ref).max() <= TOL * np.abs(ref).max()
    sim.close()


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
