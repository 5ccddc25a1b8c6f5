"""Pins of the oracle's Poisson solve, Eq. (1): lap(phi) = -rho/eps0 with Dirichlet
electrodes (cathode phi_c at z = 0, anode phi_a at z = Lz) and periodic x, y.

Checked against: the exact linear vacuum potential, second-order convergence on
a manufactured solution, a dense LU solve (numpy.linalg.solve) of an
independently assembled matrix, and symmetry of the operator.
"""
import numpy as np
import pytest

import oracle as O

EPS0 = 8.8541878128e-12


def test_vacuum_potential_is_linear():
    nx, ny, nz, h = 6, 4, 10, 3e-9
    rho = np.zeros((nz + 1, ny, nx))
    phi, it, rel = O.poisson(nx, ny, nz, h, 0.0, 3000.0, rho, rtol=1e-14)
    z = np.arange(nz + 1) * h
    expect = 3000.0 * z / (nz * h)
    assert rel <= 1e-14
    assert np.allclose(phi, expect[:, None, None], rtol=0, atol=1e-10)
    # non-zero cathode potential as well
    phi, it, rel = O.poisson(nx, ny, nz, h, -5.0, 7.0, rho, rtol=1e-14)
    expect = -5.0 + 12.0 * z / (nz * h)
    assert np.allclose(phi, expect[:, None, None], rtol=0, atol=1e-12)


def _mms(n):
    nx, ny, nz = n, n, 2 * n
    Lx = Ly = 100e-9
    Lz = 200e-9
    h = Lx / nx
    V, A = 50.0, 3.0
    x = np.arange(nx) * h
    y = np.arange(ny) * h
    z = np.arange(nz + 1) * h
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    mode = np.sin(2 * np.pi * X / Lx) * np.sin(2 * np.pi * Y / Ly) * np.sin(np.pi * Z / Lz)
    exact = V * Z / Lz + A * mode
    lam = (2 * np.pi / Lx) ** 2 + (2 * np.pi / Ly) ** 2 + (np.pi / Lz) ** 2
    rho = EPS0 * A * lam * mode  # -eps0 lap(exact)
    phi, it, rel = O.poisson(nx, ny, nz, h, 0.0, V, rho, rtol=1e-13)
    return np.abs(phi - exact).max()


def test_manufactured_solution_second_order():
    errs = [_mms(n) for n in (8, 16, 32)]
    ratios = [errs[i] / errs[i + 1] for i in range(len(errs) - 1)]
    for r in ratios:
        assert 3.6 < r < 4.4, (errs, ratios)


def _dense_matrix(nx, ny, nz):
    nu = nz - 1
    N = nx * ny * nu
    A = np.zeros((N, N))
    idx = lambda i, j, k: (k * ny + j) * nx + i
    for k in range(nu):
        for j in range(ny):
            for i in range(nx):
                r = idx(i, j, k)
                A[r, r] += 6.0
                for di, dj in ((1, 0), (-1, 0), (0, 1), (0, -1)):
                    A[r, idx((i + di) % nx, (j + dj) % ny, k)] -= 1.0
                for dk in (1, -1):
                    if 0 <= k + dk < nu:
                        A[r, idx(i, j, k + dk)] -= 1.0
    return A


@pytest.mark.parametrize("shape", [(4, 4, 8), (3, 5, 4), (4, 4, 2)])
def test_matches_dense_lu(shape):
    nx, ny, nz = shape
    h = 2e-9
    rng = np.random.default_rng(5)
    rho = rng.standard_normal((nz + 1, ny, nx)) * 1e6
    phi_c, phi_a = -2.0, 11.0
    phi, it, rel = O.poisson(nx, ny, nz, h, phi_c, phi_a, rho, rtol=1e-14)
    A = _dense_matrix(nx, ny, nz)
    b = (h * h / EPS0 * rho[1:nz]).reshape(-1).copy()
    plane = nx * ny
    b[:plane] += phi_c
    b[-plane:] += phi_a
    x = np.linalg.solve(A, b)
    assert np.allclose(phi[1:nz].reshape(-1), x, rtol=0, atol=1e-11 * np.abs(x).max())
    assert np.all(phi[0] == phi_c) and np.all(phi[nz] == phi_a)


def test_operator_is_symmetric_positive():
    nx, ny, nz = 5, 6, 9
    rng = np.random.default_rng(9)
    n = nx * ny * (nz - 1)
    x = rng.standard_normal(n)
    y = rng.standard_normal(n)
    Ax = O.laplacian_apply(nx, ny, nz, x)
    Ay = O.laplacian_apply(nx, ny, nz, y)
    assert abs(y @ Ax - x @ Ay) <= 1e-12 * abs(y @ Ax)
    assert x @ Ax > 0
    assert np.allclose(Ax, _dense_matrix(nx, ny, nz) @ x, rtol=0, atol=1e-12)
