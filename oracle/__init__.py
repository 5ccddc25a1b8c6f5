"""ctypes wrapper of the plain FP64 CPU oracle (pic_oracle.c).

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the benchmark's
CPU-baseline and reference legs are the only users. The oracle is independent of the CUDA
library (no shared source, header or helper); both sides consume the seeded
inputs of ``paper_2606_05893_gb300.workloads`` and nothing else.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pic_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
# the same source built with -fopenmp (bit-identical results, all host cores)
_LIB_OMP = os.path.join(_BUILD, "liboracle_omp.so")
_lock = threading.Lock()
_lib = None
_lib_omp = None

MAXSP = 8


class OrCfg(C.Structure):
    _fields_ = [
        ("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32),
        ("h", C.c_double), ("dt", C.c_double), ("phi_c", C.c_double), ("phi_a", C.c_double),
        ("rho_bg", C.c_double),
        ("sort_interval", C.c_int32),
        ("cg_rtol", C.c_double),
        ("cg_maxit", C.c_int32),
        ("seed", C.c_uint64),
        ("warm_zero", C.c_int32),
        ("nsp", C.c_int32),
        ("q", C.c_double * MAXSP), ("m", C.c_double * MAXSP), ("w", C.c_double * MAXSP),
        ("role", C.c_int32 * MAXSP),
        ("variable_weights", C.c_int32),
    ]


class OrMoments(C.Structure):
    _fields_ = [
        ("count", C.c_int64 * MAXSP),
        ("injected", C.c_int64 * MAXSP),
        ("abs_cathode", C.c_int64 * MAXSP), ("abs_anode", C.c_int64 * MAXSP),
        ("abs_energy_cathode", C.c_double * MAXSP), ("abs_energy_anode", C.c_double * MAXSP),
        ("n_ionization", C.c_int64), ("n_elastic", C.c_int64), ("n_suppressed", C.c_int64),
        ("step", C.c_int64),
        ("cg_iters", C.c_int32),
        ("cg_resid_rel", C.c_double),
        ("total_charge", C.c_double),
        ("kinetic", C.c_double * MAXSP),
        ("field_energy", C.c_double),
        ("charge_to_cathode_last", C.c_double), ("charge_to_anode_last", C.c_double),
        ("next_pid", C.c_uint32),
        ("anode_V", C.c_double),
        ("n_cx", C.c_int64),
    ]


def _compile(out: str, extra, force: bool) -> str:
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(_SRC):
        return out
    os.makedirs(_BUILD, exist_ok=True)
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", *extra, "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def build(force: bool = False, omp: bool = False) -> str:
    """Compile the oracle with gcc (-ffp-contract=off): single-threaded, or with
    -fopenmp (omp=True). Both builds are made by default; returns the asked one."""
    with _lock:
        _compile(_LIB, [], force)
        _compile(_LIB_OMP, ["-fopenmp"], force)
        return _LIB_OMP if omp else _LIB


def lib(omp: bool = False):
    """The serial oracle library, or its OpenMP build (omp=True)."""
    global _lib, _lib_omp
    if (_lib_omp if omp else _lib) is None:
        L = C.CDLL(build(omp=omp))
        P = C.c_void_p
        d = C.POINTER(C.c_double)
        u32 = C.POINTER(C.c_uint32)
        L.or_create.restype = P
        L.or_create.argtypes = [C.POINTER(OrCfg)]
        L.or_destroy.argtypes = [P]
        L.or_add_xsec.argtypes = [P, C.c_int, C.c_int, C.c_int, C.c_int, C.c_double, C.c_int, d, d]
        L.or_add_source.argtypes = [P, C.c_int, C.c_double, C.c_double, C.c_double, C.c_double, C.c_double]
        L.or_set_background_density.argtypes = [P, C.c_double]
        L.or_set_source.argtypes = [P, C.c_int, C.c_double, C.c_double]
        L.or_set_circuit.argtypes = [P, C.c_double, C.c_double, C.c_double]
        L.or_load.argtypes = [P, C.c_int, C.c_int64, d, d]
        L.or_load_m.argtypes = [P, C.c_int, C.c_int64, d, d, u32]
        L.or_get_multiplicity.argtypes = [P, C.c_int, u32]
        L.or_count.restype = C.c_int64
        L.or_count.argtypes = [P, C.c_int]
        L.or_get_particles.argtypes = [P, C.c_int, d, d, u32]
        L.or_set_velocities.argtypes = [P, C.c_int, d]
        L.or_get_rho.argtypes = [P, d]
        L.or_get_phi.argtypes = [P, d]
        L.or_set_phi.argtypes = [P, d]
        L.or_get_ncount.argtypes = [P, C.c_int, C.POINTER(C.c_int32)]
        L.or_get_cell_start.argtypes = [P, C.c_int, C.POINTER(C.c_int64)]
        L.or_get_log.restype = C.c_int64
        L.or_get_log.argtypes = [P, u32]
        L.or_get_hits.restype = C.c_int64
        L.or_get_hits.argtypes = [P, u32, C.POINTER(C.c_int32), u32, d, d]
        L.or_inject.restype = C.c_int64
        L.or_inject.argtypes = [P]
        L.or_sort.argtypes = [P]
        L.or_deposit.argtypes = [P]
        L.or_solve.restype = C.c_int
        L.or_solve.argtypes = [P]
        L.or_push_collide_resolve.argtypes = [P]
        L.or_step.argtypes = [P]
        L.or_step_until_solve.restype = C.c_int
        L.or_step_until_solve.argtypes = [P]
        L.or_step_finish.argtypes = [P]
        L.or_get_moments.argtypes = [P, C.POINTER(OrMoments)]
        L.or_get_step.restype = C.c_uint32
        L.or_get_step.argtypes = [P]
        L.or_set_step.argtypes = [P, C.c_uint32]
        L.or_get_next_pid.restype = C.c_uint32
        L.or_get_next_pid.argtypes = [P]
        L.or_get_source_acc.restype = C.c_double
        L.or_get_source_acc.argtypes = [P, C.c_int]
        L.or_philox.argtypes = [u32, u32, u32]
        L.or_u01.restype = C.c_double
        L.or_u01.argtypes = [C.c_uint32, C.c_uint32]
        L.or_poisson.restype = C.c_int
        L.or_poisson.argtypes = [C.c_int, C.c_int, C.c_int, C.c_double, C.c_double, C.c_double, d, d,
                                 C.c_double, C.c_int, d]
        L.or_laplacian_apply.argtypes = [C.c_int, C.c_int, C.c_int, d, d]
        L.or_deposit_points.argtypes = [C.c_int, C.c_int, C.c_int, C.c_double, C.c_int64, d, C.c_double, d]
        L.or_gather_points.argtypes = [P, C.c_int64, d, d]
        L.or_sigma.restype = C.c_double
        L.or_sigma.argtypes = [P, C.c_int, C.c_double]
        L.or_uniform_fill.argtypes = [C.c_uint64, C.c_uint32, C.c_int64, C.c_uint32, C.c_uint32, C.c_uint32, d]
        L.or_sizeof_cfg.restype = C.c_size_t
        L.or_sizeof_moments.restype = C.c_size_t
        L.or_set_threads.restype = C.c_int
        L.or_set_threads.argtypes = [C.c_int]
        assert L.or_sizeof_cfg() == C.sizeof(OrCfg), "oracle cfg layout mismatch"
        assert L.or_sizeof_moments() == C.sizeof(OrMoments), "oracle moments layout mismatch"
        if omp:
            _lib_omp = L
        else:
            _lib = L
    return _lib_omp if omp else _lib


def set_threads(n: int = 0) -> int:
    """Threads of the OpenMP build (0: all it may use); returns the count in use."""
    return int(lib(omp=True).or_set_threads(int(n)))


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def philox(ctr, key):
    """Philox4x32-10 of one counter (4 x u32) and key (2 x u32) -> 4 x u32."""
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().or_philox(c.ctypes.data_as(C.POINTER(C.c_uint32)), k.ctypes.data_as(C.POINTER(C.c_uint32)),
                    out.ctypes.data_as(C.POINTER(C.c_uint32)))
    return out


def uniforms(seed, n, step, tag, j=0, pid0=0):
    """FP64 uniforms of Philox(pid0..pid0+n-1, step, tag, j): array [n, 2]."""
    out = np.zeros(2 * n)
    lib().or_uniform_fill(seed, pid0, n, step, tag, j, _dp(out))
    return out.reshape(n, 2)


def u01(a, b):
    return lib().or_u01(int(a), int(b))


def poisson(nx, ny, nz, h, phi_c, phi_a, rho, phi0=None, rtol=1e-12, maxit=100000):
    """Solve Eq. (1) on the node grid; returns (phi over all nodes, iterations, true rel. residual)."""
    rho = np.ascontiguousarray(rho, dtype=np.float64).reshape(-1)
    nn = nx * ny * (nz + 1)
    assert rho.size == nn
    phi = np.zeros(nn) if phi0 is None else np.array(phi0, dtype=np.float64).reshape(-1).copy()
    rel = C.c_double(0.0)
    it = lib().or_poisson(nx, ny, nz, h, phi_c, phi_a, _dp(rho), _dp(phi), rtol, maxit, C.byref(rel))
    return phi.reshape(nz + 1, ny, nx), it, rel.value


def laplacian_apply(nx, ny, nz, x_interior):
    x = np.ascontiguousarray(x_interior, dtype=np.float64).reshape(-1)
    y = np.zeros_like(x)
    lib().or_laplacian_apply(nx, ny, nz, _dp(x), _dp(y))
    return y


def deposit_points(nx, ny, nz, h, xyz, qw):
    xyz = np.ascontiguousarray(xyz, dtype=np.float64).reshape(-1, 3)
    rho = np.zeros(nx * ny * (nz + 1))
    lib().or_deposit_points(nx, ny, nz, h, xyz.shape[0], _dp(xyz), qw, _dp(rho))
    return rho.reshape(nz + 1, ny, nx)


class Oracle:
    """One PIC/MCC instance on the CPU, driven step by step."""

    def __init__(self, wl, cg_rtol=None, cg_maxit=None, warm_zero=False, preload=True,
                 background_density=0.0, omp=False):
        """omp=True runs the OpenMP build of the same source (bit-identical results)."""
        L = lib(omp)
        self._L = L
        c = OrCfg()
        c.nx, c.ny, c.nz = wl.nx, wl.ny, wl.nz
        c.h, c.dt, c.phi_c, c.phi_a, c.rho_bg = wl.h, wl.dt, wl.phi_cathode, wl.phi_anode, wl.rho_background
        c.sort_interval = wl.sort_interval
        c.cg_rtol = wl.cg_rtol if cg_rtol is None else cg_rtol
        c.cg_maxit = 100000 if cg_maxit is None else cg_maxit
        c.seed = wl.seed
        c.warm_zero = 1 if warm_zero else 0
        c.nsp = len(wl.species)
        for i, s in enumerate(wl.species):
            c.q[i], c.m[i], c.w[i], c.role[i] = s.charge_C, s.mass_kg, s.weight, s.role
        c.variable_weights = 1 if getattr(wl, "variable_weights", False) else 0
        self.wl = wl
        self.nsp = c.nsp
        self._h = L.or_create(C.byref(c))
        if not self._h:
            raise ValueError("oracle rejected the configuration")
        self._keep = []
        for x in wl.xsec:
            E = np.ascontiguousarray(x.E_eV, dtype=np.float64)
            s = np.ascontiguousarray(x.sigma_m2, dtype=np.float64)
            L.or_add_xsec(self._h, x.kind, x.projectile, x.target, x.product, x.threshold_eV, E.size, _dp(E), _dp(s))
        for q in wl.sources:
            L.or_add_source(self._h, q.species, q.cx, q.cy, q.radius, q.flux_m2s, q.T_K)
        if background_density > 0:
            L.or_set_background_density(self._h, background_density)
        if preload and wl.preload:
            for sp, pre in enumerate(wl.preload):
                self.load(sp, *pre)

    def close(self):
        if self._h:
            self._L.or_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def load(self, sp, x, v, m=None):
        """Append particles (pids from the next free one); m: their multiplicities
        (variable-weight workloads), 1 each when None."""
        x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, 3)
        v = np.ascontiguousarray(v, dtype=np.float64).reshape(-1, 3)
        assert x.shape == v.shape
        if m is None:
            r = self._L.or_load(self._h, sp, x.shape[0], _dp(x), _dp(v))
        else:
            m = np.ascontiguousarray(m, dtype=np.uint32).reshape(-1)
            assert m.shape[0] == x.shape[0]
            r = self._L.or_load_m(self._h, sp, x.shape[0], _dp(x), _dp(v), m.ctypes.data_as(C.POINTER(C.c_uint32)))
        if r != 0:
            raise ValueError("bad species or multiplicities")

    def multiplicity(self, sp):
        """Multiplicities of species sp in store order (the order of particles())."""
        out = np.zeros(self.count(sp), dtype=np.uint32)
        self._L.or_get_multiplicity(self._h, sp, out.ctypes.data_as(C.POINTER(C.c_uint32)))
        return out

    def step(self, n=1):
        for _ in range(n):
            self._L.or_step(self._h)

    def step_until_solve(self):
        return self._L.or_step_until_solve(self._h)

    def step_finish(self):
        self._L.or_step_finish(self._h)

    def inject(self):
        return self._L.or_inject(self._h)

    def sort(self):
        self._L.or_sort(self._h)

    def deposit(self):
        self._L.or_deposit(self._h)

    def solve(self):
        return self._L.or_solve(self._h)

    def count(self, sp):
        return int(self._L.or_count(self._h, sp))

    def particles(self, sp):
        n = self.count(sp)
        x = np.zeros((n, 3)); v = np.zeros((n, 3)); pid = np.zeros(n, dtype=np.uint32)
        self._L.or_get_particles(self._h, sp, _dp(x), _dp(v), pid.ctypes.data_as(C.POINTER(C.c_uint32)))
        return x, v, pid

    def set_velocities(self, sp, v):
        v = np.ascontiguousarray(v, dtype=np.float64).reshape(-1, 3)
        assert v.shape[0] == self.count(sp)
        self._L.or_set_velocities(self._h, sp, _dp(v))

    def rho(self):
        wl = self.wl
        out = np.zeros(wl.nx * wl.ny * (wl.nz + 1))
        self._L.or_get_rho(self._h, _dp(out))
        return out.reshape(wl.nz + 1, wl.ny, wl.nx)

    def phi(self):
        wl = self.wl
        out = np.zeros(wl.nx * wl.ny * (wl.nz + 1))
        self._L.or_get_phi(self._h, _dp(out))
        return out.reshape(wl.nz + 1, wl.ny, wl.nx)

    def set_phi(self, phi):
        phi = np.ascontiguousarray(phi, dtype=np.float64).reshape(-1)
        self._L.or_set_phi(self._h, _dp(phi))

    def ncount(self, sp):
        wl = self.wl
        out = np.zeros(wl.nx * wl.ny * wl.nz, dtype=np.int32)
        self._L.or_get_ncount(self._h, sp, out.ctypes.data_as(C.POINTER(C.c_int32)))
        return out.reshape(wl.nz, wl.ny, wl.nx)

    def cell_start(self, sp):
        wl = self.wl
        out = np.zeros(wl.nx * wl.ny * wl.nz + 1, dtype=np.int64)
        self._L.or_get_cell_start(self._h, sp, out.ctypes.data_as(C.POINTER(C.c_int64)))
        return out

    def ionization_log(self):
        n = self._L.or_get_log(self._h, None)
        out = np.zeros((max(n, 1), 3), dtype=np.uint32)
        self._L.or_get_log(self._h, out.ctypes.data_as(C.POINTER(C.c_uint32)))
        return out[:n]

    def hits(self):
        """Ions absorbed at the cathode since the last call (the log is emptied),
        ordered by (step, pid): pid, species, step, xy (n x 2: where the path
        crossed z = 0), v (n x 3: v^{n+1/2})."""
        n = self._L.or_get_hits(self._h, None, None, None, None, None)
        m = max(n, 1)
        pid = np.zeros(m, dtype=np.uint32)
        sp = np.zeros(m, dtype=np.int32)
        step = np.zeros(m, dtype=np.uint32)
        xy = np.zeros((m, 2))
        v = np.zeros((m, 3))
        self._L.or_get_hits(self._h, pid.ctypes.data_as(C.POINTER(C.c_uint32)), sp.ctypes.data_as(C.POINTER(C.c_int32)),
                          step.ctypes.data_as(C.POINTER(C.c_uint32)), _dp(xy), _dp(v))
        o = np.lexsort((pid[:n], step[:n]))
        return {"pid": pid[:n][o], "species": sp[:n][o], "step": step[:n][o], "xy": xy[:n][o], "v": v[:n][o]}

    def gather(self, xyz):
        xyz = np.ascontiguousarray(xyz, dtype=np.float64).reshape(-1, 3)
        E = np.zeros_like(xyz)
        self._L.or_gather_points(self._h, xyz.shape[0], _dp(xyz), _dp(E))
        return E

    def sigma(self, ch, E):
        return self._L.or_sigma(self._h, ch, float(E))

    @property
    def step_index(self):
        return int(self._L.or_get_step(self._h))

    @step_index.setter
    def step_index(self, v):
        self._L.or_set_step(self._h, int(v))

    @property
    def next_pid(self):
        return int(self._L.or_get_next_pid(self._h))

    def set_circuit(self, R_ohm, C_farad, V0):
        """External RC circuit on the anode (off unless R > 0 and C > 0)."""
        self._L.or_set_circuit(self._h, float(R_ohm), float(C_farad), float(V0))

    def set_source(self, q, flux, T_K):
        if self._L.or_set_source(self._h, q, flux, T_K) != 0:
            raise ValueError("bad source")

    def source_acc(self, q):
        return self._L.or_get_source_acc(self._h, q)

    def moments(self):
        m = OrMoments()
        self._L.or_get_moments(self._h, C.byref(m))
        ns = self.nsp
        return {
            "step": m.step,
            "count": list(m.count[:ns]),
            "injected": list(m.injected[:ns]),
            "abs_cathode": list(m.abs_cathode[:ns]),
            "abs_anode": list(m.abs_anode[:ns]),
            "abs_energy_cathode": list(m.abs_energy_cathode[:ns]),
            "abs_energy_anode": list(m.abs_energy_anode[:ns]),
            "n_ionization": m.n_ionization,
            "n_elastic": m.n_elastic,
            "n_suppressed": m.n_suppressed,
            "cg_iters": m.cg_iters,
            "cg_resid_rel": m.cg_resid_rel,
            "total_charge": m.total_charge,
            "kinetic": list(m.kinetic[:ns]),
            "field_energy": m.field_energy,
            "charge_to_cathode_last": m.charge_to_cathode_last,
            "charge_to_anode_last": m.charge_to_anode_last,
            "next_pid": m.next_pid,
            "anode_V": m.anode_V,
            "n_cx": m.n_cx,
        }
