"""GB300-native electrostatic PIC/MCC library: thin Python binding of libpic_gb300.so.

The C ABI (include/pic.h) is mirrored name for name: ``pic_create``,
``pic_inject``, ``pic_inject_particles``, ``pic_step``, ``pic_moments``,
``pic_destroy`` and the inspection hooks. This module only marshals arguments
(numpy arrays, ctypes structures, the torch CUDA stream); every step of the
PIC/MCC cycle runs in the library's CUDA kernels. There is no CPU fallback:
importing the binding without the built library, or calling it without a GPU,
raises.

``Simulation`` wraps one handle built from a ``workloads.Workload``.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import workloads  # noqa: F401  (seeded input generators)

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libpic_gb300.so")

PIC_MAX_SPECIES = 8
PIC_OK, PIC_EINVAL, PIC_ENOMEM, PIC_ECAPACITY, PIC_ENOCONV, PIC_ECUDA, PIC_ETIMEOUT, PIC_ESTATE = 0, -1, -2, -3, -4, -5, -6, -7
STATUS_NAMES = {0: "PIC_OK", -1: "PIC_EINVAL", -2: "PIC_ENOMEM", -3: "PIC_ECAPACITY", -4: "PIC_ENOCONV",
                -5: "PIC_ECUDA", -6: "PIC_ETIMEOUT", -7: "PIC_ESTATE"}
PIC_ELECTRON, PIC_NEUTRAL, PIC_ION = 0, 1, 2
PIC_XS_IONIZATION, PIC_XS_ELASTIC, PIC_XS_CHARGE_EXCHANGE = 0, 1, 2
PIC_FP64, PIC_MIXED = 0, 1
PIC_WARM_PREV, PIC_WARM_ZERO, PIC_WARM_UNET = 0, 1, 2
PIC_FIELD_RHO, PIC_FIELD_PHI, PIC_FIELD_NCOUNT = 0, 1, 2


class pic_species(C.Structure):
    _fields_ = [("charge_C", C.c_double), ("mass_kg", C.c_double), ("weight", C.c_double),
                ("role", C.c_int32), ("capacity", C.c_int64)]


class pic_xsec(C.Structure):
    _fields_ = [("kind", C.c_int32), ("projectile", C.c_int32), ("target", C.c_int32), ("product", C.c_int32),
                ("threshold_eV", C.c_double), ("n", C.c_int32),
                ("E_eV", C.POINTER(C.c_double)), ("sigma_m2", C.POINTER(C.c_double))]


class pic_instance_cfg(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32),
                ("h", C.c_double), ("dt", C.c_double), ("phi_cathode_V", C.c_double), ("phi_anode_V", C.c_double),
                ("rho_background", C.c_double),
                ("sort_interval", C.c_int32),
                ("cg_rtol", C.c_double), ("cg_maxit", C.c_int32),
                ("precision", C.c_int32),
                ("seed", C.c_uint64),
                ("nspecies", C.c_int32), ("species", C.POINTER(pic_species)),
                ("nxsec", C.c_int32), ("xsec", C.POINTER(pic_xsec)),
                ("warm_start", C.c_int32),
                ("variable_weights", C.c_int32)]


class pic_moments_t(C.Structure):
    _fields_ = [("step", C.c_int64),
                ("count", C.c_int64 * PIC_MAX_SPECIES),
                ("injected", C.c_int64 * PIC_MAX_SPECIES),
                ("absorbed_cathode", C.c_int64 * PIC_MAX_SPECIES),
                ("absorbed_anode", C.c_int64 * PIC_MAX_SPECIES),
                ("absorbed_energy_cathode_J", C.c_double * PIC_MAX_SPECIES),
                ("absorbed_energy_anode_J", C.c_double * PIC_MAX_SPECIES),
                ("ionizations", C.c_int64), ("elastic", C.c_int64), ("suppressed", C.c_int64),
                ("cg_iters", C.c_int32), ("cg_resid_rel", C.c_double),
                ("total_charge_C", C.c_double),
                ("kinetic_J", C.c_double * PIC_MAX_SPECIES),
                ("field_energy_J", C.c_double),
                ("charge_to_cathode_C", C.c_double), ("charge_to_anode_C", C.c_double),
                ("next_pid", C.c_uint32), ("error_flags", C.c_int32),
                ("pushed", C.c_int64 * PIC_MAX_SPECIES),
                ("anode_V", C.c_double), ("charge_exchanges", C.c_int64)]


PHASES = ["inject", "sort", "deposit", "solve", "efield", "push_electron", "push_ion", "push_neutral", "resolve"]
PIC_NPHASES = len(PHASES)


EXPORTED = ["pic_create", "pic_inject", "pic_inject_particles", "pic_inject_particles_m", "pic_get_multiplicity",
            "pic_step", "pic_moments", "pic_destroy",
            "pic_last_error", "pic_get_count", "pic_get_particles", "pic_get_field", "pic_set_phi", "pic_solve",
            "pic_sort_now", "pic_get_cell_start", "pic_get_ionization_log", "pic_philox",
            "pic_set_mcc_background", "pic_version", "pic_set_profiling", "pic_get_phase_times",
            "pic_launch_count", "pic_kernel_count", "pic_poisson_solve_static", "pic_set_sort_interval",
            "pic_set_hit_log", "pic_get_hits", "pic_set_circuit", "pic_save", "pic_load",
            "pic_set_warm_unet", "pic_get_phi_device", "pic_set_launch_shape", "pic_set_allocator",
            "unet_num_weights", "unet_create", "unet_destroy", "unet_set_weights", "unet_get_weights",
            "unet_forward", "unet_backward", "unet_get_grads", "unet_train_step", "unet_last_error",
            "unet_launch_count", "unet_make_sample", "unet_layer_forward", "unet_layer_backward",
            "unet_train_step_residual", "unet_set_profiling", "unet_get_layer_times"]

_lib = None


class PicError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def load_library(path: str = None):
    """Load libpic_gb300.so (built by ``_build.build()``); raises if it is missing.
    PIC_GB300_LIB names another build of the same library to load instead (the
    checked build, ``_build.build(checked=True)``); the first load of a process
    decides."""
    global _lib
    if _lib is not None:
        return _lib
    if path is None:
        path = os.environ.get("PIC_GB300_LIB") or LIB_PATH
    if not os.path.exists(path):
        raise ImportError(f"libpic_gb300.so not built ({path}); run __graft_entry__.build() or "
                          "python -m paper_2606_05893_gb300._build")
    L = C.CDLL(path)
    P = C.c_void_p
    d = C.POINTER(C.c_double)
    u32 = C.POINTER(C.c_uint32)
    i64 = C.POINTER(C.c_int64)
    st = C.c_int
    sig = {
        "pic_create": ([C.POINTER(pic_instance_cfg), C.c_int32, P, C.POINTER(P)], st),
        "pic_inject": ([P, C.c_int32, C.c_int32, C.c_double, C.c_double, C.c_double, C.c_double, C.c_double], st),
        "pic_inject_particles": ([P, C.c_int32, C.c_int32, C.c_int64, d, d], st),
        "pic_inject_particles_m": ([P, C.c_int32, C.c_int32, C.c_int64, d, d, u32], st),
        "pic_get_multiplicity": ([P, C.c_int32, C.c_int32, C.c_int64, i64, u32], st),
        "pic_step": ([P, C.c_int32], st),
        "pic_moments": ([P, C.c_int32, C.POINTER(pic_moments_t)], st),
        "pic_destroy": ([P], st),
        "pic_last_error": ([P], C.c_char_p),
        "pic_get_count": ([P, C.c_int32, C.c_int32, i64], st),
        "pic_get_particles": ([P, C.c_int32, C.c_int32, C.c_int64, i64, u32, d, d], st),
        "pic_get_field": ([P, C.c_int32, C.c_int32, C.c_int32, P], st),
        "pic_set_phi": ([P, C.c_int32, d], st),
        "pic_solve": ([P, C.c_int32, d, d, C.POINTER(C.c_int32), d], st),
        "pic_sort_now": ([P, C.c_int32], st),
        "pic_get_cell_start": ([P, C.c_int32, C.c_int32, i64], st),
        "pic_get_ionization_log": ([P, C.c_int32, C.c_int64, i64, u32], st),
        "pic_philox": ([P, C.c_int64, u32, u32, u32], st),
        "pic_set_mcc_background": ([P, C.c_int32, C.c_double], st),
        "pic_set_sort_interval": ([P, C.c_int32, C.c_int32], st),
        "pic_set_launch_shape": ([P, C.c_int32, C.c_int32], st),
        "pic_set_allocator": ([P, P, P], st),
        "pic_set_hit_log": ([P, C.c_int32, C.c_int64], st),
        "pic_set_circuit": ([P, C.c_int32, C.c_double, C.c_double, C.c_double], st),
        "pic_save": ([P, C.c_int32, C.c_char_p], st),
        "pic_load": ([P, C.c_int32, C.c_char_p], st),
        "pic_get_hits": ([P, C.c_int32, C.c_int64, i64, i64, C.POINTER(C.c_uint32), C.POINTER(C.c_int32), i64,
                          d, d, d], st),
        "pic_version": ([], C.c_char_p),
        "pic_set_profiling": ([P, C.c_int32], st),
        "pic_get_phase_times": ([P, C.c_int32, d, i64], st),
        "pic_launch_count": ([], C.c_uint64),
        "pic_kernel_count": ([], C.c_uint64),
        "pic_poisson_solve_static": ([C.c_int32, C.c_int32, C.c_int32, C.c_double, C.c_double, C.c_double, P, P,
                                      C.c_double, C.c_int32, P, C.POINTER(C.c_int32), d], st),
        "pic_set_warm_unet": ([P, C.c_int32, P], st),
        "pic_get_phi_device": ([P, C.c_int32, P], st),
        "unet_num_weights": ([], C.c_int64),
        "unet_create": ([C.c_int32, C.c_int32, C.c_int32, P, C.POINTER(P)], st),
        "unet_destroy": ([P], st),
        "unet_set_weights": ([P, C.POINTER(C.c_float), C.c_int64], st),
        "unet_get_weights": ([P, C.POINTER(C.c_float), C.c_int64], st),
        "unet_forward": ([P, P, P], st),
        "unet_backward": ([P, P], st),
        "unet_get_grads": ([P, C.POINTER(C.c_float), C.c_int64], st),
        "unet_train_step": ([P, P, P, C.c_int32, C.c_float, d], st),
        "unet_last_error": ([P], C.c_char_p),
        "unet_launch_count": ([], C.c_uint64),
        "unet_make_sample": ([P, P, P, P, P, d], st),
        "unet_layer_forward": ([P, C.c_int32, P, P, C.c_int32], st),
        "unet_train_step_residual": ([P, P, C.c_float, d], st),
        "unet_set_profiling": ([P, C.c_int32], st),
        "unet_get_layer_times": ([P, d, i64], st),
        "unet_layer_backward": ([P, C.c_int32, P, P, P, C.POINTER(C.c_float), C.c_int64], st),
    }
    for name, (args, res) in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res
    _lib = L
    return L


def _i64p(a):
    return a.ctypes.data_as(C.POINTER(C.c_int64))


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _check(h, status):
    if status != PIC_OK:
        msg = load_library().pic_last_error(h)
        raise PicError(status, msg.decode() if msg else "")
    return status


# ----------------------------------------------------------------------------
# name-for-name wrappers of the C ABI
# ----------------------------------------------------------------------------
def pic_create(cfgs, stream=None):
    """cfgs: list of pic_instance_cfg (their arrays must stay alive during the call)."""
    L = load_library()
    arr = (pic_instance_cfg * len(cfgs))(*cfgs)
    h = C.c_void_p()
    if stream is None:
        stream = _torch_stream()
    _check(None, L.pic_create(arr, len(cfgs), C.c_void_p(stream), C.byref(h)))
    return h


def pic_inject(h, inst, species, cx, cy, radius_m, flux_m2s, T_K):
    return _check(h, load_library().pic_inject(h, inst, species, cx, cy, radius_m, flux_m2s, T_K))


def pic_inject_particles(h, inst, species, x, v):
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, 3)
    v = np.ascontiguousarray(v, dtype=np.float64).reshape(-1, 3)
    if x.shape != v.shape:
        raise ValueError("x and v must have the same shape [n, 3]")
    return _check(h, load_library().pic_inject_particles(h, inst, species, x.shape[0], _dp(x), _dp(v)))


def pic_inject_particles_m(h, inst, species, x, v, mw):
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, 3)
    v = np.ascontiguousarray(v, dtype=np.float64).reshape(-1, 3)
    mw = np.ascontiguousarray(mw, dtype=np.uint32).reshape(-1)
    if x.shape != v.shape or mw.shape[0] != x.shape[0]:
        raise ValueError("x, v must have the shape [n, 3] and mw [n]")
    return _check(h, load_library().pic_inject_particles_m(h, inst, species, x.shape[0], _dp(x), _dp(v),
                                                           mw.ctypes.data_as(C.POINTER(C.c_uint32))))


def pic_get_multiplicity(h, inst, species):
    n = pic_get_count(h, inst, species)
    mw = np.zeros(max(n, 1), dtype=np.uint32)
    got = C.c_int64()
    _check(h, load_library().pic_get_multiplicity(h, inst, species, mw.shape[0], C.byref(got),
                                                  mw.ctypes.data_as(C.POINTER(C.c_uint32))))
    return mw[:got.value]


def pic_step(h, nsteps=1, check=True):
    s = load_library().pic_step(h, nsteps)
    return _check(h, s) if check else s


def pic_moments(h, inst=0):
    m = pic_moments_t()
    _check(h, load_library().pic_moments(h, inst, C.byref(m)))
    return m


def pic_destroy(h):
    if h:
        load_library().pic_destroy(h)


def pic_last_error(h):
    r = load_library().pic_last_error(h)
    return r.decode() if r else ""


def pic_version():
    return load_library().pic_version().decode()


def pic_get_count(h, inst, species):
    n = C.c_int64()
    _check(h, load_library().pic_get_count(h, inst, species, C.byref(n)))
    return n.value


def pic_get_particles(h, inst, species):
    n = pic_get_count(h, inst, species)
    cap = max(n, 1)
    pid = np.zeros(cap, dtype=np.uint32)
    x = np.zeros((cap, 3))
    v = np.zeros((cap, 3))
    got = C.c_int64()
    _check(h, load_library().pic_get_particles(h, inst, species, cap, C.byref(got),
                                               pid.ctypes.data_as(C.POINTER(C.c_uint32)), _dp(x), _dp(v)))
    k = got.value
    return x[:k], v[:k], pid[:k]


def pic_get_field(h, inst, which, shape, species=0):
    dtype = np.int32 if which == PIC_FIELD_NCOUNT else np.float64
    out = np.zeros(shape, dtype=dtype)
    _check(h, load_library().pic_get_field(h, inst, which, species, out.ctypes.data_as(C.c_void_p)))
    return out


def pic_set_phi(h, inst, phi):
    phi = np.ascontiguousarray(phi, dtype=np.float64)
    return _check(h, load_library().pic_set_phi(h, inst, _dp(phi)))


def pic_solve(h, inst, rho, phi0):
    rho = np.ascontiguousarray(rho, dtype=np.float64)
    phi = np.array(phi0, dtype=np.float64, copy=True, order="C")
    it = C.c_int32()
    rel = C.c_double()
    s = load_library().pic_solve(h, inst, _dp(rho), _dp(phi), C.byref(it), C.byref(rel))
    _check(h, s)
    return phi, it.value, rel.value


def pic_sort_now(h, inst=0):
    return _check(h, load_library().pic_sort_now(h, inst))


def pic_get_cell_start(h, inst, species, ncell):
    out = np.zeros(ncell + 1, dtype=np.int64)
    _check(h, load_library().pic_get_cell_start(h, inst, species, out.ctypes.data_as(C.POINTER(C.c_int64))))
    return out


def pic_get_ionization_log(h, inst=0, cap=1 << 20):
    rows = np.zeros((cap, 3), dtype=np.uint32)
    n = C.c_int64()
    _check(h, load_library().pic_get_ionization_log(h, inst, cap, C.byref(n),
                                                    rows.ctypes.data_as(C.POINTER(C.c_uint32))))
    return rows[: n.value].copy()


def pic_philox(h, n, ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4 * n, dtype=np.uint32)
    _check(h, load_library().pic_philox(h, n, c.ctypes.data_as(C.POINTER(C.c_uint32)),
                                        k.ctypes.data_as(C.POINTER(C.c_uint32)),
                                        out.ctypes.data_as(C.POINTER(C.c_uint32))))
    return out.reshape(n, 4)


def pic_set_mcc_background(h, inst, density):
    return _check(h, load_library().pic_set_mcc_background(h, inst, density))


def pic_set_circuit(h, inst, R_ohm, C_farad, V0):
    return _check(h, load_library().pic_set_circuit(h, inst, float(R_ohm), float(C_farad), float(V0)))


def pic_save(h, inst, path):
    return _check(h, load_library().pic_save(h, inst, os.fsencode(path)))


def pic_load(h, inst, path):
    return _check(h, load_library().pic_load(h, inst, os.fsencode(path)))


def pic_set_hit_log(h, inst, capacity):
    return _check(h, load_library().pic_set_hit_log(h, inst, capacity))


def pic_get_hits(h, inst=0, cap=1 << 16):
    """Ions absorbed at the cathode since the last read, ordered by (step, pid):
    a dict of pid, species, step, x (n x 3, z = 0), v (n x 3), ke_eV, and lost."""
    n, lost = C.c_int64(), C.c_int64()
    pid = np.zeros(max(cap, 1), dtype=np.uint32)
    sp = np.zeros(max(cap, 1), dtype=np.int32)
    step = np.zeros(max(cap, 1), dtype=np.int64)
    x = np.zeros((max(cap, 1), 3))
    v = np.zeros((max(cap, 1), 3))
    ke = np.zeros(max(cap, 1))
    _check(h, load_library().pic_get_hits(h, inst, cap, C.byref(n), C.byref(lost),
                                          pid.ctypes.data_as(C.POINTER(C.c_uint32)),
                                          sp.ctypes.data_as(C.POINTER(C.c_int32)), _i64p(step), _dp(x), _dp(v),
                                          _dp(ke)))
    k = n.value
    return {"pid": pid[:k].copy(), "species": sp[:k].copy(), "step": step[:k].copy(), "x": x[:k].copy(),
            "v": v[:k].copy(), "ke_eV": ke[:k].copy(), "lost": lost.value}


def pic_set_sort_interval(h, inst, interval):
    return _check(h, load_library().pic_set_sort_interval(h, inst, interval))


def pic_set_launch_shape(h, inst, blocks_per_sm):
    return _check(h, load_library().pic_set_launch_shape(h, inst, blocks_per_sm))


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)
_allocator = None  # the registered callbacks, kept alive while the library may call them


def pic_set_allocator(alloc=None, free=None):
    """Route the library's device memory through Python callables alloc(nbytes) -> int
    pointer (0 on failure) and free(ptr); both None restores cudaMalloc / cudaFree.
    Only while no PIC or U-Net handle is alive (PicError otherwise)."""
    global _allocator
    if (alloc is None) != (free is None):
        raise ValueError("give both alloc and free, or neither")
    if alloc is None:
        _check(None, load_library().pic_set_allocator(None, None, None))
        _allocator = None
        return
    a = ALLOC_FN(lambda nbytes, ctx: alloc(int(nbytes)) or None)
    f = FREE_FN(lambda ptr, ctx: free(int(ptr)))
    _check(None, load_library().pic_set_allocator(C.cast(a, C.c_void_p), C.cast(f, C.c_void_p), None))
    _allocator = (a, f)


def use_torch_allocator(enable=True):
    """Back the library's device memory by PyTorch's caching allocator (its
    blocks count in torch.cuda.memory_allocated), or restore cudaMalloc."""
    if not enable:
        return pic_set_allocator()
    import torch

    def alloc(nbytes):
        try:
            return torch.cuda.caching_allocator_alloc(nbytes)
        except RuntimeError:
            return 0

    return pic_set_allocator(alloc, torch.cuda.caching_allocator_delete)


def pic_set_profiling(h, on=True):
    return _check(h, load_library().pic_set_profiling(h, 1 if on else 0))


def pic_get_phase_times(h, inst=0):
    ms = np.zeros(PIC_NPHASES)
    cnt = np.zeros(PIC_NPHASES, dtype=np.int64)
    _check(h, load_library().pic_get_phase_times(h, inst, _dp(ms), cnt.ctypes.data_as(C.POINTER(C.c_int64))))
    return {name: (float(ms[i]), int(cnt[i])) for i, name in enumerate(PHASES)}


def pic_launch_count():
    return int(load_library().pic_launch_count())


def pic_kernel_count():
    return int(load_library().pic_kernel_count())


PIC_STATIC_MAX_UNKNOWNS = 1 << 18


def pic_poisson_solve_static(nx, ny, nz, h, phi_cathode_V, phi_anode_V, rho_dev_ptr, phi_dev_ptr, rtol, maxit,
                             stream=None):
    """No-allocation Poisson solve on caller-owned device buffers (raw pointers,
    e.g. torch tensor data_ptr()). Returns (status, iterations, relative residual)."""
    if stream is None:
        stream = _torch_stream()
    it = C.c_int32()
    rel = C.c_double()
    st = load_library().pic_poisson_solve_static(nx, ny, nz, h, phi_cathode_V, phi_anode_V, C.c_void_p(rho_dev_ptr),
                                                 C.c_void_p(phi_dev_ptr), rtol, maxit, C.c_void_p(stream),
                                                 C.byref(it), C.byref(rel))
    return st, it.value, rel.value


# ----------------------------------------------------------------------------
# learned warm start (include/unet.h): device buffers are passed as raw device
# pointers (e.g. torch tensor data_ptr()); weights as flat FP32 host arrays
# ----------------------------------------------------------------------------
# The library's network (layer table of csrc/unet_api.cu): the 3x3x3 convolutions
# in the order e0a e0b e1a e1b e2a e2b e3a e3b d2a d2b d1a d1b d0a d0b as
# (name, input channels, output channels), then the 1x1x1 output layer.
UNET_LAYERS = (("e0a", 2, 16), ("e0b", 16, 16), ("e1a", 16, 32), ("e1b", 32, 32), ("e2a", 32, 64),
               ("e2b", 64, 64), ("e3a", 64, 128), ("e3b", 128, 128), ("d2a", 192, 64), ("d2b", 64, 64),
               ("d1a", 96, 32), ("d1b", 32, 32), ("d0a", 48, 16), ("d0b", 16, 16))
UNET_WEIGHT_SHAPES = [(co, ci, 3, 3, 3) for _, ci, co in UNET_LAYERS] + [(1, 16)]


def _ucheck(net, status):
    if status != PIC_OK:
        msg = load_library().unet_last_error(net)
        raise PicError(status, msg.decode() if msg else "")
    return status


def unet_num_weights():
    return int(load_library().unet_num_weights())


def unet_create(D, H, W, stream=None):
    if stream is None:
        stream = _torch_stream()
    net = C.c_void_p()
    st = load_library().unet_create(D, H, W, C.c_void_p(stream), C.byref(net))
    if st != PIC_OK:
        raise PicError(st, f"unet_create({D}, {H}, {W})")
    return net


def unet_destroy(net):
    if net:
        load_library().unet_destroy(net)


def _fp(a):
    return a.ctypes.data_as(C.POINTER(C.c_float))


def unet_set_weights(net, w):
    w = np.ascontiguousarray(w, dtype=np.float32).reshape(-1)
    return _ucheck(net, load_library().unet_set_weights(net, _fp(w), w.size))


def unet_get_weights(net):
    w = np.zeros(unet_num_weights(), dtype=np.float32)
    _ucheck(net, load_library().unet_get_weights(net, _fp(w), w.size))
    return w


def unet_get_grads(net):
    g = np.zeros(unet_num_weights(), dtype=np.float32)
    _ucheck(net, load_library().unet_get_grads(net, _fp(g), g.size))
    return g


def unet_forward(net, x_ptr, y_ptr):
    return _ucheck(net, load_library().unet_forward(net, C.c_void_p(x_ptr), C.c_void_p(y_ptr)))


def unet_backward(net, dy_ptr):
    return _ucheck(net, load_library().unet_backward(net, C.c_void_p(dy_ptr)))


def unet_train_step(net, x_ptr, t_ptr, loss_planes, lr):
    loss = C.c_double()
    _ucheck(net, load_library().unet_train_step(net, C.c_void_p(x_ptr), C.c_void_p(t_ptr), loss_planes, lr,
                                                C.byref(loss)))
    return loss.value


def unet_train_step_residual(net, x_ptr, lr):
    loss = C.c_double()
    _ucheck(net, load_library().unet_train_step_residual(net, C.c_void_p(x_ptr), lr, C.byref(loss)))
    return loss.value


def unet_make_sample(net, phi_new_ptr, phi_old_ptr, x_ptr, t_ptr):
    s = C.c_double()
    _ucheck(net, load_library().unet_make_sample(net, C.c_void_p(phi_new_ptr), C.c_void_p(phi_old_ptr),
                                                 C.c_void_p(x_ptr), C.c_void_p(t_ptr), C.byref(s)))
    return s.value


def unet_layer_forward(net, layer, x_ptr, y_ptr, relu=False):
    return _ucheck(net, load_library().unet_layer_forward(net, layer, C.c_void_p(x_ptr), C.c_void_p(y_ptr),
                                                          1 if relu else 0))


def unet_layer_backward(net, layer, x_ptr, dz_ptr, dx_ptr, n_dw):
    dw = np.zeros(n_dw, dtype=np.float32)
    _ucheck(net, load_library().unet_layer_backward(net, layer, C.c_void_p(x_ptr), C.c_void_p(dz_ptr),
                                                    C.c_void_p(dx_ptr) if dx_ptr else None, _fp(dw), n_dw))
    return dw


def unet_set_profiling(net, on=True):
    return _ucheck(net, load_library().unet_set_profiling(net, 1 if on else 0))


def unet_get_layer_times(net):
    """Per convolution (UNET_LAYERS order): (summed forward ms, timed launches)."""
    ms = np.zeros(len(UNET_LAYERS))
    cnt = np.zeros(len(UNET_LAYERS), dtype=np.int64)
    _ucheck(net, load_library().unet_get_layer_times(net, _dp(ms), cnt.ctypes.data_as(C.POINTER(C.c_int64))))
    return {name: (float(ms[i]), int(cnt[i])) for i, (name, _, _) in enumerate(UNET_LAYERS)}


def unet_launch_count():
    return int(load_library().unet_launch_count())


def pic_set_warm_unet(h, inst, net):
    return _check(h, load_library().pic_set_warm_unet(h, inst, net if net else None))


def pic_get_phi_device(h, inst, dev_ptr):
    return _check(h, load_library().pic_get_phi_device(h, inst, C.c_void_p(dev_ptr)))


class UNet:
    """One network (include/unet.h) for D x H x W volumes; torch CUDA tensors as
    device buffers."""

    def __init__(self, D, H, W, weights=None, stream=None):
        import torch
        self.D, self.H, self.W = D, H, W
        self.net = unet_create(D, H, W, stream)
        self.y = torch.zeros((D, H, W), dtype=torch.float32, device="cuda")
        if weights is not None:
            self.set_weights(weights)

    def close(self):
        if self.net:
            unet_destroy(self.net)
            self.net = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_weights(self, w):
        unet_set_weights(self.net, w)

    def weights(self):
        return unet_get_weights(self.net)

    def grads(self):
        return unet_get_grads(self.net)

    @staticmethod
    def _dev(t, dtype, shape, what):
        """The device pointer of a contiguous CUDA tensor of the given dtype and shape (the
        library reads raw memory: a wrong dtype or shape is refused, not reinterpreted)."""
        import torch
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.is_contiguous()):
            raise TypeError(f"{what}: a contiguous CUDA tensor is required")
        if t.dtype != dtype or tuple(t.shape) != tuple(shape):
            raise TypeError(f"{what}: expected {dtype} of shape {tuple(shape)}, got {t.dtype} {tuple(t.shape)}")
        return t.data_ptr()

    def forward(self, x):
        """x: CUDA float32 tensor (2, D, H, W); returns a (D, H, W) tensor (the network's own buffer)."""
        import torch
        unet_forward(self.net, self._dev(x, torch.float32, (2, self.D, self.H, self.W), "x"), self.y.data_ptr())
        return self.y

    def backward(self, dy):
        import torch
        unet_backward(self.net, self._dev(dy, torch.float32, (self.D, self.H, self.W), "dy"))
        return self.grads()

    def train_step(self, x, t, lr, loss_planes=None):
        import torch
        return unet_train_step(self.net, self._dev(x, torch.float32, (2, self.D, self.H, self.W), "x"),
                               self._dev(t, torch.float32, (self.D, self.H, self.W), "t"),
                               self.D - 1 if loss_planes is None else loss_planes, lr)

    def train_step_residual(self, x, lr):
        """Adam step on the residual the warm start leaves (unet_train_step_residual)."""
        import torch
        return unet_train_step_residual(self.net, self._dev(x, torch.float32, (2, self.D, self.H, self.W), "x"), lr)

    def make_sample(self, phi_new, phi_old, x, t):
        import torch
        nodes = (self.D + 1) * self.H * self.W
        pn = self._dev(phi_new.reshape(-1), torch.float64, (nodes,), "phi_new")
        po = self._dev(phi_old.reshape(-1), torch.float64, (nodes,), "phi_old")
        return unet_make_sample(self.net, pn, po, self._dev(x, torch.float32, (2, self.D, self.H, self.W), "x"),
                                self._dev(t, torch.float32, (self.D, self.H, self.W), "t"))


def _torch_stream():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("the PIC/MCC library needs a CUDA GPU; none is visible")
    return torch.cuda.current_stream().cuda_stream


# ----------------------------------------------------------------------------
# convenience: one handle built from a workload
# ----------------------------------------------------------------------------
class _CfgHolder:
    """Keeps the ctypes arrays a pic_instance_cfg points to alive."""

    def __init__(self, wl, precision, cg_rtol, cg_maxit, warm_start, sort_interval):
        sp = (pic_species * len(wl.species))()
        for i, s in enumerate(wl.species):
            sp[i].charge_C, sp[i].mass_kg, sp[i].weight = s.charge_C, s.mass_kg, s.weight
            sp[i].role, sp[i].capacity = s.role, int(s.capacity)
        self.tables = []
        xs = (pic_xsec * max(len(wl.xsec), 1))()
        for i, x in enumerate(wl.xsec):
            E = np.ascontiguousarray(x.E_eV, dtype=np.float64)
            s = np.ascontiguousarray(x.sigma_m2, dtype=np.float64)
            self.tables += [E, s]
            xs[i].kind, xs[i].projectile, xs[i].target, xs[i].product = x.kind, x.projectile, x.target, x.product
            xs[i].threshold_eV, xs[i].n = x.threshold_eV, E.size
            xs[i].E_eV, xs[i].sigma_m2 = _dp(E), _dp(s)
        c = pic_instance_cfg()
        c.nx, c.ny, c.nz = wl.nx, wl.ny, wl.nz
        c.h, c.dt, c.phi_cathode_V, c.phi_anode_V = wl.h, wl.dt, wl.phi_cathode, wl.phi_anode
        c.rho_background = wl.rho_background
        c.sort_interval = wl.sort_interval if sort_interval is None else sort_interval
        c.cg_rtol = wl.cg_rtol if cg_rtol is None else cg_rtol
        c.cg_maxit = wl.cg_maxit if cg_maxit is None else cg_maxit
        c.precision = precision
        c.seed = wl.seed
        c.nspecies = len(wl.species)
        c.species = sp
        c.nxsec = len(wl.xsec)
        c.xsec = xs
        c.warm_start = warm_start
        c.variable_weights = 1 if getattr(wl, "variable_weights", False) else 0
        self.sp, self.xs, self.cfg = sp, xs, c


class Simulation:
    """One or more instances of the GB300 PIC/MCC step driven through the C ABI."""

    def __init__(self, workloads_, precision=PIC_FP64, cg_rtol=None, cg_maxit=None, warm_start=PIC_WARM_PREV,
                 preload=True, sort_interval=None, stream=None, background_density=0.0):
        if not isinstance(workloads_, (list, tuple)):
            workloads_ = [workloads_]
        self.wls = list(workloads_)
        self.wl = self.wls[0]
        self._holders = [_CfgHolder(w, precision, cg_rtol, cg_maxit, warm_start, sort_interval) for w in self.wls]
        self.h = pic_create([hd.cfg for hd in self._holders], stream)
        for i, w in enumerate(self.wls):
            for q in w.sources:
                pic_inject(self.h, i, q.species, q.cx, q.cy, q.radius, q.flux_m2s, q.T_K)
            if background_density > 0:
                pic_set_mcc_background(self.h, i, background_density)
            if preload and w.preload:
                for sp, pre in enumerate(w.preload):
                    if not len(pre[0]):
                        continue
                    if len(pre) == 3:  # with multiplicities
                        pic_inject_particles_m(self.h, i, sp, pre[0], pre[1], pre[2])
                    else:
                        pic_inject_particles(self.h, i, sp, pre[0], pre[1])

    def save(self, path, inst=0):
        """Checkpoint of one instance (pic_save)."""
        pic_save(self.h, inst, path)

    def load(self, path, inst=0):
        """Resume one instance from a checkpoint (pic_load)."""
        pic_load(self.h, inst, path)

    def close(self):
        if self.h:
            pic_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, n=1, check=True):
        return pic_step(self.h, n, check)

    def moments(self, inst=0):
        m = pic_moments(self.h, inst)
        ns = len(self.wls[inst].species)
        return {
            "step": m.step, "count": list(m.count[:ns]), "injected": list(m.injected[:ns]),
            "abs_cathode": list(m.absorbed_cathode[:ns]), "abs_anode": list(m.absorbed_anode[:ns]),
            "abs_energy_cathode": list(m.absorbed_energy_cathode_J[:ns]),
            "abs_energy_anode": list(m.absorbed_energy_anode_J[:ns]),
            "n_ionization": m.ionizations, "n_elastic": m.elastic, "n_suppressed": m.suppressed,
            "cg_iters": m.cg_iters, "cg_resid_rel": m.cg_resid_rel, "total_charge": m.total_charge_C,
            "kinetic": list(m.kinetic_J[:ns]), "field_energy": m.field_energy_J,
            "charge_to_cathode_last": m.charge_to_cathode_C, "charge_to_anode_last": m.charge_to_anode_C,
            "next_pid": m.next_pid, "error_flags": m.error_flags, "pushed": list(m.pushed[:ns]), "anode_V": m.anode_V,
            "n_cx": m.charge_exchanges,
        }

    def particles(self, sp, inst=0):
        return pic_get_particles(self.h, inst, sp)

    def multiplicity(self, sp, inst=0):
        return pic_get_multiplicity(self.h, inst, sp)

    def count(self, sp, inst=0):
        return pic_get_count(self.h, inst, sp)

    def rho(self, inst=0):
        w = self.wls[inst]
        return pic_get_field(self.h, inst, PIC_FIELD_RHO, (w.nz + 1, w.ny, w.nx))

    def phi(self, inst=0):
        w = self.wls[inst]
        return pic_get_field(self.h, inst, PIC_FIELD_PHI, (w.nz + 1, w.ny, w.nx))

    def set_phi(self, phi, inst=0):
        pic_set_phi(self.h, inst, phi)

    def ncount(self, sp, inst=0):
        w = self.wls[inst]
        return pic_get_field(self.h, inst, PIC_FIELD_NCOUNT, (w.nz, w.ny, w.nx), species=sp)

    def cell_start(self, sp, inst=0):
        w = self.wls[inst]
        return pic_get_cell_start(self.h, inst, sp, w.nx * w.ny * w.nz)

    def sort_now(self, inst=0):
        pic_sort_now(self.h, inst)

    def solve(self, rho, phi0=None, inst=0):
        w = self.wls[inst]
        if phi0 is None:
            phi0 = np.zeros((w.nz + 1, w.ny, w.nx))
        return pic_solve(self.h, inst, rho, phi0)

    def ionization_log(self, inst=0):
        return pic_get_ionization_log(self.h, inst)
