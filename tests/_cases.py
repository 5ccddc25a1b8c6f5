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


def cathode_hits_case(n_ions=40, n_other=20, kmax=12, seed=11):
    """Field-free box (both electrodes at 0 V, weight 1e-30) with ions heading
    for the cathode: ion i starts at z0 = (k_i + 1/2) |vz| dt, k_i in [0, kmax),
    with a large transverse speed, some of them next to the x = Lx face so that
    the crossing point wraps. Electrons and neutrals head for the cathode too.
    Returns the workload and the per-ion k_i."""
    wl = bare(nx=4, ny=4, nz=16, h=5e-9, dt=1e-16)
    rng = np.random.default_rng(seed)
    Lx, Ly, _ = wl.L
    k = rng.integers(0, kmax, n_ions)
    vz = -rng.uniform(2e4, 2e5, n_ions)
    vxy = rng.uniform(-2e6, 2e6, (n_ions, 2))
    x0 = rng.random((n_ions, 2)) * np.array([Lx, Ly])
    x0[: n_ions // 4, 0] = Lx - 1e-10
    vxy[: n_ions // 4, 0] = 2e6
    z0 = (k + 0.5) * (-vz) * wl.dt
    xi = np.column_stack([x0, z0])
    vi = np.column_stack([vxy, vz])
    xo = np.column_stack([rng.random((n_other, 2)) * np.array([Lx, Ly]), rng.uniform(1e-12, 2e-11, n_other)])
    ve = np.column_stack([np.zeros((n_other, 2)), -rng.uniform(1e5, 1e6, n_other)])
    vn = np.column_stack([np.zeros((n_other, 2)), -rng.uniform(2e5, 1e6, n_other)])
    wl.preload = [(xo, ve), (xo.copy(), vn), (xi, vi)]
    return wl, k


def cx_xsec(sigma, ion=2, neutral=1, E=None):
    """Resonant charge exchange of species `ion` on `neutral` (the ion leaves as a
    neutral of the same element); constant sigma, or a table over E (eV)."""
    if E is None:
        return W.XSec(W.XS_CHARGE_EXCHANGE, ion, neutral, neutral, 0.0, np.array([1.0]), np.array([sigma]))
    return W.XSec(W.XS_CHARGE_EXCHANGE, ion, neutral, neutral, 0.0, np.asarray(E, float), np.asarray(sigma, float))


def cx_cells_case(seed=21, sigma_cx=1e-10, sigma_ion=None, capacity=1 << 14, with_electrons=False, n_dense_i=60,
                  n_dense_n=90):
    """Ions and neutrals (weight 1, both electrodes at 0 V) in a few cells: a cell
    with more neutrals than ions, one with more ions than neutrals, one with
    ions only, one with neutrals only. sigma_cx = 1e-10 m^2 makes
    u dt n sigma >= 1e2 for every ion (P = 1 in FP64). With electrons, each ion
    cell also holds 100 eV electrons (ionization with the same huge sigma when
    sigma_ion is given), which compete for the same victims."""
    xs = [cx_xsec(sigma_cx)]
    if sigma_ion is not None:
        xs.append(const_xsec(W.XS_IONIZATION, sigma_ion, threshold=W.CU_IONIZATION_EV))
    wl = bare(nx=8, ny=8, nz=8, h=5e-9, dt=1e-16, weight=1.0, capacity=capacity, seed=seed, xsec=xs)
    rng = np.random.default_rng(seed)
    h = wl.h

    def in_cell(n, c):
        return (np.array(c) + 0.05 + 0.9 * rng.random((n, 3))) * h

    cells = [((2, 3, 4), n_dense_i, n_dense_n), ((5, 5, 5), 70, 7), ((1, 6, 2), 30, 0), ((6, 1, 3), 0, 40)]
    xi = np.concatenate([in_cell(ni, c) for c, ni, _ in cells if ni])
    xn = np.concatenate([in_cell(nn, c) for c, _, nn in cells if nn])
    vi = isotropic(rng, xi.shape[0], 1.0e4) * rng.uniform(0.5, 1.5, (xi.shape[0], 1))
    vn = rng.standard_normal(xn.shape) * 500.0
    if with_electrons:
        xe = np.concatenate([in_cell(25, c) for c, ni, _ in cells if ni])
        ve = isotropic(rng, xe.shape[0], speed_of_eV(100.0))
    else:
        xe, ve = np.zeros((0, 3)), np.zeros((0, 3))
    wl.preload = [(xe, ve), (xn, vn), (xi, vi)]
    return wl


def weighted_ionization_case(seed=3, m_e=(1, 4), m_n=(1, 4), E_eV=100.0, sigma_ion=1e-17, n_dense_e=300,
                             n_dense_n=400):
    """ionization_cells_case with variable weights: every electron and neutral
    carries a multiplicity drawn uniformly from the given inclusive range, and
    every ion the multiplicity of the electron it sits on (zero net charge at
    t = 0)."""
    wl = ionization_cells_case(seed=seed, sigma_ion=sigma_ion, E_eV=E_eV, n_dense_e=n_dense_e, n_dense_n=n_dense_n)
    wl.variable_weights = True
    rng = np.random.default_rng(seed + 1000)
    (xe, ve), (xn, vn), (xi, vi) = wl.preload
    me = rng.integers(m_e[0], m_e[1] + 1, xe.shape[0]).astype(np.uint32)
    mn = rng.integers(m_n[0], m_n[1] + 1, xn.shape[0]).astype(np.uint32)
    wl.preload = [(xe, ve, me), (xn, vn, mn), (xi, vi, me.copy())]
    return wl


def with_multiplicities(wl, lo=1, hi=4, seed=0):
    """The same workload with variable weights: each preloaded particle gets a
    multiplicity drawn uniformly from [lo, hi]."""
    wl.variable_weights = True
    rng = np.random.default_rng(seed)
    wl.preload = [(p[0], p[1], rng.integers(lo, hi + 1, p[0].shape[0]).astype(np.uint32)) for p in wl.preload]
    return wl
