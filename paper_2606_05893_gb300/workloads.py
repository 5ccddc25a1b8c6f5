"""Seeded synthetic workloads for the electrostatic PIC/MCC cycle.

This module only *generates inputs*: grid/physics configurations, preloaded
particle populations, surface sources and cross-section tables. It contains
none of the PIC/MCC step arithmetic, so both the CUDA library and the CPU
oracle may consume what it produces without sharing any method code.

The paper runs its plasma domain with particles injected from the cathode
(emitted electrons, evaporated/sputtered Cu neutrals; PIC/MCC paragraph and
Appendix A) and ionizing collisions e + Cu -> 2e + Cu+ (Eq. 4). It publishes no
PIC dataset, so the populations below are synthetic stand-ins with the shapes of
that workload: an electron beam column above an emitter patch, a Cu vapour cloud
concentrated over the same patch, and a minority of Cu+ ions.

All random numbers here come from numpy's PCG64 generator seeded by the caller.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np

# CODATA 2018 constants (SI)
E_CHARGE = 1.602176634e-19
M_E = 9.1093837015e-31
EPS0 = 8.8541878128e-12
K_B = 1.380649e-23
AMU = 1.66053906660e-27
M_CU = 63.546 * AMU

ELECTRON, NEUTRAL, ION = 0, 1, 2
XS_IONIZATION, XS_ELASTIC, XS_CHARGE_EXCHANGE = 0, 1, 2

# Lotz single-shell ionization constants for Cu (a: generic Lotz constant,
# q: electrons in the outer shell, P: first ionization energy of Cu).
LOTZ_A_CM2_EV2 = 4.5e-14
LOTZ_Q = 1
CU_IONIZATION_EV = 7.73
ELASTIC_SIGMA_M2 = 1e-19


@dataclasses.dataclass
class Species:
    name: str
    charge_C: float
    mass_kg: float
    weight: float
    role: int
    capacity: int


@dataclasses.dataclass
class XSec:
    kind: int
    projectile: int
    target: int
    product: int
    threshold_eV: float
    E_eV: np.ndarray
    sigma_m2: np.ndarray


@dataclasses.dataclass
class Source:
    species: int
    cx: float
    cy: float
    radius: float
    flux_m2s: float
    T_K: float


@dataclasses.dataclass
class Workload:
    name: str
    nx: int
    ny: int
    nz: int
    h: float
    dt: float
    phi_cathode: float
    phi_anode: float
    species: List[Species]
    xsec: List[XSec]
    sources: List[Source]
    seed: int
    sort_interval: int = 20
    cg_rtol: float = 1e-8
    cg_maxit: int = 200
    rho_background: float = 0.0
    # preloaded particles per species: (x[n,3], v[n,3]) float64, or with
    # variable weights (x, v, m[n]) with m the integer multiplicities
    preload: Optional[list] = None
    steps: int = 1000
    # particles carry integer multiplicities (each stands for m x the species
    # weight); events between unequal multiplicities split the heavier partner
    variable_weights: bool = False

    @property
    def L(self):
        return (self.nx * self.h, self.ny * self.h, self.nz * self.h)

    def n_particles(self):
        if not self.preload:
            return 0
        return int(sum(p[0].shape[0] for p in self.preload))

    def n_physical(self):
        """Physical particles the preload stands for, per species (multiplicity x weight)."""
        if not self.preload:
            return [0.0] * len(self.species)
        return [float((p[2].sum() if len(p) > 2 else p[0].shape[0]) * sp.weight)
                for p, sp in zip(self.preload, self.species)]


def lotz_table(n: int = 2048, E_max: float = 1e5, P: float = CU_IONIZATION_EV):
    """Lotz-form ionization cross-section sigma(E) = a q ln(E/P) / (E P) for E > P.

    Tabulated at n points uniform in ln E over [P, E_max]. Returns (E_eV, sigma_m2).
    """
    E = P * np.exp(np.linspace(0.0, math.log(E_max / P), n))
    E[0] = P
    a_m2 = LOTZ_A_CM2_EV2 * 1e-4
    with np.errstate(divide="ignore", invalid="ignore"):
        sig = a_m2 * LOTZ_Q * np.log(E / P) / (E * P)
    sig[0] = 0.0
    sig = np.maximum(sig, 0.0)
    return E.astype(np.float64), sig.astype(np.float64)


def cu_plasma_species(weight: float, capacity: int):
    return [
        Species("e", -E_CHARGE, M_E, weight, ELECTRON, capacity),
        Species("Cu", 0.0, M_CU, weight, NEUTRAL, capacity),
        Species("Cu+", E_CHARGE, M_CU, weight, ION, capacity),
    ]


def cu_plasma_xsec(n_table: int = 2048):
    E, s = lotz_table(n_table)
    return [
        XSec(XS_IONIZATION, 0, 1, 2, CU_IONIZATION_EV, E, s),
        XSec(XS_ELASTIC, 0, 1, 1, 0.0, np.array([1.0]), np.array([ELASTIC_SIGMA_M2])),
    ]


def _maxwellian(rng, n, T_K, m):
    s = math.sqrt(K_B * T_K / m)
    return rng.standard_normal((n, 3)) * s


def preload_cu_plasma(rng, n_total, L, cx, cy, r_emit, field_Vm, mix=(0.6, 0.3, 0.1),
                      e_layout="cylinder", T_e_eV=0.5, T_cu_K=2000.0):
    """Synthetic initial population (electrons, Cu, Cu+).

    Electrons: uniform in a cylinder of radius r_emit above the emitter over the
    whole gap (e_layout='cylinder') or uniform over the box (e_layout='box');
    0.5 eV Maxwellian plus the drift speed sqrt(2 e F z / m_e) an electron
    leaving the cathode at rest would have at height z in the applied field F.
    Cu and Cu+: radial Gaussian (sigma_r = r_emit) about the emitter centre,
    half-normal in z with sigma_z = 2 r_emit (redrawn until inside the gap);
    2000 K Maxwellian.
    """
    Lx, Ly, Lz = L
    ne = int(round(n_total * mix[0]))
    nn = int(round(n_total * mix[1]))
    ni = int(n_total - ne - nn)
    out = []
    # electrons
    if e_layout == "cylinder":
        r = r_emit * np.sqrt(rng.random(ne))
        th = 2 * math.pi * rng.random(ne)
        x = np.stack([cx + r * np.cos(th), cy + r * np.sin(th), rng.random(ne) * Lz], axis=1)
    else:
        x = rng.random((ne, 3)) * np.array([Lx, Ly, Lz])
    v = _maxwellian(rng, ne, T_e_eV * E_CHARGE / K_B, M_E)
    v[:, 2] += np.sqrt(2.0 * E_CHARGE * max(field_Vm, 0.0) * x[:, 2] / M_E)
    out.append((x, v))
    for n in (nn, ni):
        xy = rng.standard_normal((n, 2)) * r_emit + np.array([cx, cy])
        z = np.abs(rng.standard_normal(n)) * 2 * r_emit
        bad = z >= Lz
        while bad.any():
            z[bad] = np.abs(rng.standard_normal(int(bad.sum()))) * 2 * r_emit
            bad = z >= Lz
        x = np.concatenate([xy, z[:, None]], axis=1)
        out.append((x, _maxwellian(rng, n, T_cu_K, M_CU)))
    for x, _ in out:
        x[:, 0] = np.mod(x[:, 0], Lx)
        x[:, 1] = np.mod(x[:, 1], Ly)
        # np.mod can return exactly L for tiny negative inputs
        x[:, 0][x[:, 0] >= Lx] = 0.0
        x[:, 1][x[:, 1] >= Ly] = 0.0
    return out


def _neutralising_weight(field, L, n_e, n_i, frac=0.1):
    """Weight making the preload's net charge produce at most `frac` of the applied field."""
    Lx, Ly, _ = L
    net = abs(n_e - n_i)
    if net == 0:
        return 1.0
    return frac * field * EPS0 * Lx * Ly / (E_CHARGE * net)


def config_small(seed: int = 42, anode_V: float = 3000.0, n_preload: int = 10_000,
                 weight: float = 100.0, e_layout: str = "box", capacity: int = 1 << 16):
    """32x32x64 cells of 5 nm, dt 0.5 fs, ~1e4 macroparticles at weight 100.

    Electron disk source R = 10 nm at the cathode centre, J = 1e12 A/m^2, 0.5 eV;
    Cu disk source 1e27 m^-2 s^-1 at 2000 K; Lotz ionization + constant elastic.
    """
    nx, ny, nz, h = 32, 32, 64, 5e-9
    L = (nx * h, ny * h, nz * h)
    cx, cy = L[0] / 2, L[1] / 2
    rng = np.random.default_rng(seed)
    field = anode_V / L[2]
    pre = preload_cu_plasma(rng, n_preload, L, cx, cy, 10e-9, field, e_layout=e_layout)
    sp = cu_plasma_species(weight, capacity)
    src = [Source(0, cx, cy, 10e-9, 1e12 / E_CHARGE, 0.5 * E_CHARGE / K_B),
           Source(1, cx, cy, 10e-9, 1e27, 2000.0)]
    return Workload("32x32x64 h=5nm N=1e4 fp64", nx, ny, nz, h, 0.5e-15, 0.0, anode_V, sp,
                    cu_plasma_xsec(), src, seed, sort_interval=20, preload=pre, steps=1000)


def config_scale(seed: int = 0, n_preload: int = 10_000_000, nx: int = 128, ny: int = 128,
                 nz: int = 256, h: float = 2.5e-9, anode_V: Optional[float] = None,
                 r_emit: float = 40e-9, capacity_factor: float = 1.25, weight: Optional[float] = None,
                 neutral_flux: float = 1e28):
    """The at-scale workload: 128x128x256 cells of 2.5 nm, emitter radius 40 nm,
    J drawn uniformly in [5e11, 5e12] A/m^2 from the seed, neutral flux 1e28,
    ~1e7 macroparticles (60% e, 30% Cu, 10% Cu+), sort every 20 steps.
    Applied field 9.375 GV/m (6 kV over 640 nm at the default grid).
    Other grid sizes keep the field (anode_V scales with the gap)."""
    L = (nx * h, ny * h, nz * h)
    field = 9.375e9
    if anode_V is None:
        anode_V = field * L[2]
    else:
        field = anode_V / L[2]
    cx, cy = L[0] / 2, L[1] / 2
    rng = np.random.default_rng(seed)
    J = 5e11 + (5e12 - 5e11) * rng.random()
    pre = preload_cu_plasma(rng, n_preload, L, cx, cy, r_emit, field, e_layout="cylinder")
    ne, ni = pre[0][0].shape[0], pre[2][0].shape[0]
    w = weight if weight is not None else _neutralising_weight(field, L, ne, ni)
    cap = int(max(1024, capacity_factor * max(p[0].shape[0] for p in pre)))
    sp = cu_plasma_species(w, cap)
    src = [Source(0, cx, cy, r_emit, J / E_CHARGE, 0.5 * E_CHARGE / K_B),
           Source(1, cx, cy, r_emit, neutral_flux, 2000.0)]
    return Workload(f"{nx}x{ny}x{nz} h={h*1e9:g}nm N={n_preload:.0e}", nx, ny, nz, h, 0.5e-15,
                    0.0, anode_V, sp, cu_plasma_xsec(), src, seed, sort_interval=20,
                    preload=pre, steps=2000)


def config_c2(seed: int = 0, n_preload: int = 10_000_000):
    return config_scale(seed=seed, n_preload=n_preload)


def config_mixed_large(seed: int = 0, n_preload: int = 50_000_000):
    """256x256x512 cells of 1.25 nm (same box as the 128^2x256 case), ~5e7 particles."""
    return config_scale(seed=seed, n_preload=n_preload, nx=256, ny=256, nz=512, h=1.25e-9)


def config_mixed_subcase(seed: int = 0):
    """64x64x128 cells at h = 1.25 nm, 0.75 kV (same field), ~7.8e5 particles."""
    return config_scale(seed=seed, n_preload=781_250, nx=64, ny=64, nz=128, h=1.25e-9)


def config_tiny(seed: int = 1, nx=8, ny=8, nz=16, h=5e-9, n_preload=600, anode_V=300.0,
                weight=1e-3, capacity=4096):
    """Tiny case for fast unit/parity tests (several tiles and a ragged tail still)."""
    L = (nx * h, ny * h, nz * h)
    cx, cy = L[0] / 2, L[1] / 2
    rng = np.random.default_rng(seed)
    field = anode_V / L[2]
    pre = preload_cu_plasma(rng, n_preload, L, cx, cy, L[0] / 4, field, e_layout="box")
    sp = cu_plasma_species(weight, capacity)
    # ~1.6 macroparticles per step from each disk at w = 1e-3
    src = [Source(0, cx, cy, L[0] / 4, 1e28, 0.5 * E_CHARGE / K_B),
           Source(1, cx, cy, L[0] / 4, 1e28, 2000.0)]
    return Workload(f"tiny {nx}x{ny}x{nz}", nx, ny, nz, h, 0.5e-15, 0.0, anode_V, sp,
                    cu_plasma_xsec(256), src, seed, sort_interval=4, preload=pre, steps=10)


def config_ensemble(seed: int = 0, n_instances: int = 48, sides=(32, 64, 96, 128), h: float = 2.5e-9):
    """Batched ensemble of independent instances of uneven sizes: grid (n, n, 2n)
    with n drawn from `sides`, applied field uniform in [5, 15] GV/m, emitter
    radius uniform in [5, 40] nm, preloaded macroparticles log-uniform in
    [1e4, 2e6], J per instance as in the at-scale workload."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n_instances):
        n = int(rng.choice(np.asarray(sides)))
        field = rng.uniform(5e9, 15e9)
        r_emit = rng.uniform(5e-9, 40e-9)
        npre = int(round(math.exp(rng.uniform(math.log(1e4), math.log(2e6)))))
        wl = config_scale(seed=seed * 1000 + i, n_preload=npre, nx=n, ny=n, nz=2 * n, h=h,
                          anode_V=field * 2 * n * h, r_emit=r_emit)
        # small populations under a wide, dense emitter are dominated by what is
        # injected: room for 200 steps of the electron source on top of the preload
        src = wl.sources[0]
        inj = src.flux_m2s * math.pi * src.radius ** 2 * wl.dt / wl.species[0].weight
        extra = int(200 * inj)
        for sp in wl.species:
            sp.capacity += extra
        out.append(wl)
    return out


def config_warm_start(seed: int = 0, n_preload: int = 10_000_000, nx: int = 128, ny: int = 128, nz: int = 256,
                      h: float = 2.5e-9, capacity_factor: float = 1.25, r_emit: float = 40e-9):
    """A run for the learned warm start's samples: the at-scale physics on the
    128x128x256 grid with the applied field uniform in [5, 15] GV/m, J uniform
    in [5e11, 5e12] A/m^2 (as the at-scale workload) and the Cu flux log-uniform
    in [1e26, 1e28] m^-2 s^-1, all drawn from the seed (emitter radius 40 nm as at
    scale; smaller boxes take a smaller one so injection stays a small fraction
    of the population per step)."""
    rng = np.random.default_rng(10_000 + seed)
    field = rng.uniform(5e9, 15e9)
    flux = math.exp(rng.uniform(math.log(1e26), math.log(1e28)))
    return config_scale(seed=seed, n_preload=n_preload, nx=nx, ny=ny, nz=nz, h=h, anode_V=field * nz * h,
                        neutral_flux=flux, capacity_factor=capacity_factor, r_emit=r_emit)
