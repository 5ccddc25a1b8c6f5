"""Pins of the oracle's cloud-in-cell deposition (charge source of Eq. 1).

rho_node = sum_p q w S(x_p - x_node) / h^3 with the trilinear hat S. Checked
against: exact total charge, a particle on a node, a particle at a cell centre,
periodic wrap, and a brute-force evaluation of the hat functions over every node.
"""
import numpy as np

import oracle as O


def test_total_charge_is_conserved():
    nx, ny, nz, h = 6, 5, 7, 1e-8
    rng = np.random.default_rng(3)
    n = 5000
    xyz = rng.random((n, 3)) * np.array([nx, ny, nz]) * h
    qw = -1.602176634e-19 * 37.0
    rho = O.deposit_points(nx, ny, nz, h, xyz, qw)  # qw = q * w; rho is charge per volume
    total = rho.sum() * h ** 3
    assert abs(total - n * qw) <= 1e-13 * abs(n * qw)


def test_particle_on_node_and_cell_centre():
    nx, ny, nz, h = 4, 4, 4, 1.0
    rho = O.deposit_points(nx, ny, nz, h, np.array([[1.0, 2.0, 3.0]]), 1.0)
    expect = np.zeros((nz + 1, ny, nx))
    expect[3, 2, 1] = 1.0
    assert np.array_equal(rho, expect)
    rho = O.deposit_points(nx, ny, nz, h, np.array([[1.5, 2.5, 0.5]]), 8.0)
    expect = np.zeros((nz + 1, ny, nx))
    for k in (0, 1):
        for j in (2, 3):
            for i in (1, 2):
                expect[k, j, i] = 1.0
    assert np.array_equal(rho, expect)


def test_periodic_wrap_in_x_and_y():
    nx, ny, nz, h = 4, 3, 2, 1.0
    rho = O.deposit_points(nx, ny, nz, h, np.array([[3.75, 2.5, 1.0]]), 1.0)
    # x: 0.25 to node 3, 0.75 to node 0 (wrapped); y: 0.5 to node 2 and node 0 (wrapped)
    expect = np.zeros((nz + 1, ny, nx))
    expect[1, 2, 3] = 0.25 * 0.5
    expect[1, 2, 0] = 0.75 * 0.5
    expect[1, 0, 3] = 0.25 * 0.5
    expect[1, 0, 0] = 0.75 * 0.5
    assert np.allclose(rho, expect, rtol=0, atol=1e-15)


def test_brute_force_hat_functions():
    nx, ny, nz, h = 4, 4, 4, 2.5e-9
    rng = np.random.default_rng(11)
    n = 200
    xyz = rng.random((n, 3)) * np.array([nx, ny, nz]) * h
    qw = 3.0e-21
    rho = O.deposit_points(nx, ny, nz, h, xyz, qw)
    L = np.array([nx, ny, nz]) * h
    brute = np.zeros((nz + 1, ny, nx))
    for k in range(nz + 1):
        for j in range(ny):
            for i in range(nx):
                node = np.array([i, j, k]) * h
                d = xyz - node
                # minimum image in the periodic directions
                d[:, 0] -= L[0] * np.round(d[:, 0] / L[0])
                d[:, 1] -= L[1] * np.round(d[:, 1] / L[1])
                hat = np.prod(np.maximum(0.0, 1.0 - np.abs(d) / h), axis=1)
                brute[k, j, i] = qw * hat.sum() / h ** 3
    assert np.allclose(rho, brute, rtol=1e-12, atol=1e-12 * np.abs(brute).max())
