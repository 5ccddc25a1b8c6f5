"""Small hand-built workloads shared by the oracle pins and the GPU parity tests.

Inputs only (geometry, species, particle arrays); no step arithmetic.
"""
import math

import numpy as np

from paper_2606_05893_gb300 import workloads as W


def bare(nx=4, ny=4, nz=16, h=5e-9, dt=1e-16, phi_c=0.0, phi_a=0.0, weight=1e-30, capacity=1 << 14,
         seed=5, xsec=None, sources=None, rho_background=0.0, sort_interval=0, cg_rtol=1e-13):
    sp = W.cu_plasma_species(weight, capacity)
    return W.Workload("bare", nx, ny, nz, h, dt, phi_c, phi_a, sp, xsec or [], sources or [], seed,
                      sort_interval=sort_interval, cg_rtol=cg_rtol, rho_background=rho_background,
                      preload=[(np.zeros((0, 3)), np.zeros((0, 3))) for _ in range(3)])


def isotropic(rng, n, speed):
    v = rng.standard_normal((n, 3))
    v /= np.linalg.norm(v, axis=1)[:, None]
    return v * speed


def speed_of_eV(E_eV, m=W.M_E):
    return math.sqrt(2.0 * E_eV * W.E_CHARGE / m)


def const_xsec(kind, sigma, threshold=0.0, target=1, product=2):
    return W.XSec(kind, 0, target, product, threshold, np.array([1.0]), np.array([sigma]))


def ionization_cells_case(seed=3, sigma_ion=1e-17, sigma_el=1e-19, E_eV=100.0, capacity=1 << 14, n_dense_e=300,
                          n_dense_n=400):
    """Electrons co-located with ions (zero net charge at t = 0, so the first push
    sees no field) in a few cells holding neutrals: one dense cell (no
    suppression) and one cell with two neutrals (most ionizations suppressed)."""
    wl = bare(nx=8, ny=8, nz=8, h=5e-9, dt=1e-16, weight=1.0, capacity=capacity, seed=seed,
              xsec=[const_xsec(W.XS_IONIZATION, sigma_ion, threshold=W.CU_IONIZATION_EV),
                    const_xsec(W.XS_ELASTIC, sigma_el, target=1, product=1)])
    rng = np.random.default_rng(seed)
    h = wl.h

    def in_cell(n, c):
        return (np.array(c) + 0.05 + 0.9 * rng.random((n, 3))) * h

    dense, sparse = (2, 3, 4), (5, 5, 5)
    xe = np.concatenate([in_cell(n_dense_e, dense), in_cell(200, sparse)])
    ve = isotropic(rng, xe.shape[0], speed_of_eV(E_eV))
    xn = np.concatenate([in_cell(n_dense_n, dense), in_cell(2, sparse)])
    vn = rng.standard_normal(xn.shape) * 500.0
    xi = xe.copy()
    vi = np.zeros_like(xi)
    wl.preload = [(xe, ve), (xn, vn), (xi, vi)]
    return wl
