"""Thin ctypes binding of the C ABI in include/clb.h (libclb.so).

Argument marshalling only: every step of the method runs in the CUDA
kernels of libclb.so.  Names mirror the C entry points; a failing call
raises ClbError with the library's message.  There is no CPU fallback: if
the library cannot be loaded or no CUDA device is present, loading fails
loudly.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

from . import build as _build

CLB_OK = 0
CLB_ERR_ARG = -1
CLB_ERR_CUDA = -2
CLB_ERR_OOM = -3
CLB_ERR_UNSTABLE = -4
CLB_ERR_STATE = -5
CLB_ERR_TIMEOUT = -6
CLB_BATCH_GRAPH, CLB_BATCH_PERSISTENT = 0, 1
W, E, S, N = 0, 1, 2, 3
CLB_PERIODIC, CLB_WALL = 0, 1
CLB_ADIABATIC, CLB_ISOTHERMAL = 0, 1
CLB_F64 = 0
CLB_F16S = 1
CLB_F16N = 2


class ClbError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"[{code}] {msg}")
        self.code = code


class ClbParams(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("forchheimer", ctypes.c_int32), ("shift", ctypes.c_int32), ("reserved", ctypes.c_int32)] + \
               [(n, ctypes.c_double) for n in ("Ra", "Da", "Pr", "J", "Gamma", "sigma", "Ma", "L", "nu",
                                               "dT", "T0", "T_init", "ax", "ay", "varpi", "s3", "s4", "sb")]


class ClbBc(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32 * 4), ("u", ctypes.c_double * 4), ("v", ctypes.c_double * 4),
                ("thermal", ctypes.c_int32 * 4), ("T", ctypes.c_double * 4)]


class ClbLattice(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in ("sb", "sv", "zeta_a", "nu", "nu_e", "alpha", "alpha_e", "K",
                                                "gbeta", "L")] + [("pitch", ctypes.c_int64)]


_lib = None

_DP = ctypes.POINTER(ctypes.c_double)
_VP = ctypes.c_void_p


def load(build_if_needed: bool = True):
    """Load libclb.so (building it first if its sources are newer)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.build() if build_if_needed else _build.LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library {path} is missing; run paper_2110_05943_gb300.build.build()")
    L = ctypes.CDLL(path)
    L.clb_params_default.argtypes = [ctypes.POINTER(ClbParams)]
    L.clb_params_default.restype = None
    L.clb_bc_cavity.argtypes = [ctypes.POINTER(ClbBc), ctypes.c_double, ctypes.c_double]
    L.clb_bc_cavity.restype = None
    L.clb_init.argtypes = [ctypes.POINTER(_VP), ctypes.POINTER(ClbParams), _DP, _DP, ctypes.POINTER(ClbBc), _VP]
    L.clb_step.argtypes = [_VP, ctypes.c_int64]
    L.clb_set_fields.argtypes = [_VP, _DP, _DP, _DP, _DP]
    L.clb_macros.argtypes = [_VP, _DP, _DP, _DP, _DP]
    L.clb_macros_device.argtypes = [_VP, _VP, _VP, _VP, _VP]
    L.clb_nusselt.argtypes = [_VP, ctypes.c_int32, _DP]
    L.clb_residual.argtypes = [_VP, _DP, _DP]
    L.clb_time.argtypes = [_VP]
    L.clb_time.restype = ctypes.c_int64
    L.clb_lattice_params.argtypes = [_VP, ctypes.POINTER(ClbLattice)]
    L.clb_state_bytes.argtypes = [_VP]
    L.clb_state_bytes.restype = ctypes.c_size_t
    L.clb_get_state.argtypes = [_VP, _VP, ctypes.c_size_t]
    L.clb_set_state.argtypes = [_VP, _VP, ctypes.c_size_t]
    L.clb_sync.argtypes = [_VP]
    L.clb_destroy.argtypes = [_VP]
    L.clb_destroy.restype = None
    L.clb_last_error.argtypes = [_VP]
    L.clb_last_error.restype = ctypes.c_char_p
    L.clb_nusselt_field_static.argtypes = [_VP, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_double,
                                           ctypes.c_double, _VP, _VP]
    L.clb_batch_init.argtypes = [ctypes.POINTER(_VP), ctypes.c_int32, ctypes.POINTER(ClbParams),
                                 ctypes.POINTER(_DP), ctypes.POINTER(ClbBc), _VP]
    L.clb_batch_step.argtypes = [_VP, ctypes.c_int64]
    L.clb_batch_set_active.argtypes = [_VP, ctypes.POINTER(ctypes.c_int32)]
    L.clb_batch_tune.argtypes = [_VP, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32)]
    L.clb_batch_set_tiling.argtypes = [_VP, ctypes.c_int32]
    L.clb_batch_set_mode.argtypes = [_VP, ctypes.c_int32]
    L.clb_batch_barrier_selftest.argtypes = [_VP, ctypes.c_int64]
    L.clb_batch_nusselt.argtypes = [_VP, ctypes.c_int32, _DP]
    L.clb_batch_macros.argtypes = [_VP, ctypes.c_int32, _DP, _DP, _DP, _DP]
    L.clb_batch_nodes.argtypes = [_VP]
    L.clb_batch_nodes.restype = ctypes.c_int64
    L.clb_batch_time.argtypes = [_VP]
    L.clb_batch_time.restype = ctypes.c_int64
    L.clb_batch_sync.argtypes = [_VP]
    L.clb_batch_last_error.argtypes = [_VP]
    L.clb_batch_last_error.restype = ctypes.c_char_p
    L.clb_batch_destroy.argtypes = [_VP]
    L.clb_batch_destroy.restype = None
    for name in ("clb_batch_init", "clb_batch_step", "clb_batch_set_active", "clb_batch_tune", "clb_batch_nusselt",
                 "clb_batch_macros", "clb_batch_sync", "clb_batch_set_tiling", "clb_batch_set_mode",
                 "clb_batch_barrier_selftest"):
        getattr(L, name).restype = ctypes.c_int
    L.clb_fp64_special_check.argtypes = [_VP, ctypes.c_int64, _VP, _VP]
    L.clb_set_tma.argtypes = [_VP, ctypes.c_int32]
    L.clb_tma_selftest.argtypes = [_VP, ctypes.c_int64]
    for name in ("clb_set_tma", "clb_tma_selftest", "clb_fp64_special_check", "clb_nusselt_field_static", "clb_init", "clb_step", "clb_set_fields", "clb_macros", "clb_macros_device", "clb_nusselt",
                 "clb_residual", "clb_lattice_params", "clb_get_state", "clb_set_state", "clb_sync"):
        getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


def _check(rc: int, h=None):
    if rc != CLB_OK:
        msg = load().clb_last_error(h)
        raise ClbError(rc, msg.decode() if msg else "")


def _dp(a):
    return None if a is None else a.ctypes.data_as(_DP)


def _f64(a, n=None):
    if a is None:
        return None
    a = np.ascontiguousarray(a, dtype=np.float64)
    if n is not None and a.size != n:
        raise ValueError(f"expected {n} values, got {a.size}")
    return a


# ------------------------------------------------------------ entry points
def clb_params_default(**overrides) -> ClbParams:
    p = ClbParams()
    load().clb_params_default(ctypes.byref(p))
    for k, v in overrides.items():
        if not hasattr(p, k):
            raise AttributeError(f"clb_params has no field {k!r}")
        setattr(p, k, int(v) if k in ("nx", "ny", "precision", "forchheimer", "shift") else float(v))
    return p


def clb_bc_cavity(Th: float = 1.0, Tc: float = 0.0) -> ClbBc:
    bc = ClbBc()
    load().clb_bc_cavity(ctypes.byref(bc), Th, Tc)
    return bc


def clb_bc(kind, u=(0.0,) * 4, v=(0.0,) * 4, T=(None,) * 4) -> ClbBc:
    """Boundary spec from per-side lists (W, E, S, N); T[s] = None means adiabatic."""
    bc = ClbBc()
    for s in range(4):
        k = kind[s]
        bc.kind[s] = CLB_WALL if k in ("wall", CLB_WALL) else CLB_PERIODIC
        bc.u[s] = float(u[s])
        bc.v[s] = float(v[s])
        bc.thermal[s] = CLB_ADIABATIC if T[s] is None else CLB_ISOTHERMAL
        bc.T[s] = 0.0 if T[s] is None else float(T[s])
    return bc


def clb_init(p: ClbParams, phi, bc: ClbBc, ay_row=None, stream=None):
    """Returns an opaque handle (int).  `stream` is a cudaStream_t as int
    (e.g. torch.cuda.current_stream().cuda_stream) or None."""
    n = p.nx * p.ny
    phi = _field(phi, n)
    ay = _field(ay_row, p.ny)
    h = _VP()
    rc = load().clb_init(ctypes.byref(h), ctypes.byref(p), _dp(phi), _dp(ay), ctypes.byref(bc),
                         _VP(stream) if stream else None)
    _check(rc, None)
    return h.value


def clb_step(h, n: int):
    _check(load().clb_step(h, int(n)), h)


def _field(a, n):
    """Scalar -> n copies; array -> flattened (ny, nx) row-major values."""
    if a is None:
        return None
    a = np.asarray(a, dtype=np.float64)
    if a.ndim == 0:
        return np.full(n, float(a))
    return _f64(a.reshape(-1), n)


def clb_set_fields(h, nx: int, ny: int, rho, ux, uy, T):
    n = nx * ny
    rho, ux, uy, T = (_field(a, n) for a in (rho, ux, uy, T))
    _check(load().clb_set_fields(h, _dp(rho), _dp(ux), _dp(uy), _dp(T)), h)


def clb_macros(h, nx: int, ny: int):
    out = [np.empty((ny, nx)) for _ in range(4)]
    _check(load().clb_macros(h, *[_dp(a) for a in out]), h)
    return tuple(out)


def clb_macros_device(h, rho_ptr=None, ux_ptr=None, uy_ptr=None, T_ptr=None):
    _check(load().clb_macros_device(h, rho_ptr, ux_ptr, uy_ptr, T_ptr), h)


def clb_nusselt(h, side: int) -> float:
    v = ctypes.c_double()
    _check(load().clb_nusselt(h, int(side), ctypes.byref(v)), h)
    return v.value


def clb_nusselt_field_static(T_ptr: int, nx: int, ny: int, side: int, L: float, dT: float, nu_ptr: int,
                             stream=None):
    """Allocation-free Nusselt reduction over a device temperature field
    (device pointers as ints); the result lands in the device double at
    nu_ptr, asynchronously on `stream`."""
    rc = load().clb_nusselt_field_static(T_ptr, int(nx), int(ny), int(side), float(L), float(dT), nu_ptr,
                                         _VP(stream) if stream else None)
    _check(rc, None)


def clb_fp64_special_check(x_ptr: int, n: int, out_ptr: int, stream=None):
    """Step's and IEEE reciprocal / square root of n device doubles (see clb.h)."""
    _check(load().clb_fp64_special_check(x_ptr, int(n), out_ptr, _VP(stream) if stream else None), None)


def clb_residual(h):
    a, b = ctypes.c_double(), ctypes.c_double()
    _check(load().clb_residual(h, ctypes.byref(a), ctypes.byref(b)), h)
    return a.value, b.value


def clb_time(h) -> int:
    return int(load().clb_time(h))


def clb_lattice_params(h) -> ClbLattice:
    lat = ClbLattice()
    _check(load().clb_lattice_params(h, ctypes.byref(lat)), h)
    return lat


def clb_get_state(h) -> bytes:
    nb = load().clb_state_bytes(h)
    buf = ctypes.create_string_buffer(nb)
    _check(load().clb_get_state(h, buf, nb), h)
    return buf.raw


def clb_set_state(h, state: bytes):
    buf = ctypes.create_string_buffer(state, len(state))
    _check(load().clb_set_state(h, buf, len(state)), h)


def clb_sync(h):
    _check(load().clb_sync(h), h)


def clb_set_tma(h, enable: bool):
    _check(load().clb_set_tma(h, int(bool(enable))), h)


def clb_tma_selftest(h, limit_cycles: int) -> int:
    """Status of the TMA-fed step's expiry check (CLB_ERR_TIMEOUT expected,
    see clb.h); the simulation's state is unchanged."""
    return load().clb_tma_selftest(h, int(limit_cycles))


def clb_destroy(h):
    if h:
        load().clb_destroy(h)


# ------------------------------------------------------------ convenience
@dataclass
class Simulation:
    """Owns one handle; fields come back as (ny, nx) numpy arrays."""
    params: ClbParams
    handle: int

    @classmethod
    def create(cls, params: ClbParams, phi, bc: ClbBc, ay_row=None, stream=None):
        return cls(params, clb_init(params, phi, bc, ay_row, stream))

    @property
    def shape(self):
        return self.params.ny, self.params.nx

    def step(self, n: int):
        clb_step(self.handle, n)

    def macros(self):
        return clb_macros(self.handle, self.params.nx, self.params.ny)

    def set_fields(self, rho, ux, uy, T):
        clb_set_fields(self.handle, self.params.nx, self.params.ny, rho, ux, uy, T)

    def nusselt(self, side: int = W) -> float:
        return clb_nusselt(self.handle, side)

    def residual(self):
        return clb_residual(self.handle)

    @property
    def time(self) -> int:
        return clb_time(self.handle)

    @property
    def lattice(self) -> ClbLattice:
        return clb_lattice_params(self.handle)

    def get_state(self) -> bytes:
        return clb_get_state(self.handle)

    def set_state(self, s: bytes):
        clb_set_state(self.handle, s)

    def sync(self):
        clb_sync(self.handle)

    def set_tma(self, enable: bool):
        clb_set_tma(self.handle, enable)

    def close(self):
        if self.handle:
            clb_destroy(self.handle)
            self.handle = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------ batches
def _bcheck(rc: int, b=None):
    if rc != CLB_OK:
        msg = load().clb_batch_last_error(b)
        raise ClbError(rc, msg.decode() if msg else "")


def clb_batch_init(params, phis, bcs, stream=None):
    """params, phis, bcs: per-case lists (phi scalar or (ny, nx) array)."""
    n = len(params)
    P = (ClbParams * n)(*params)
    B = (ClbBc * n)(*bcs)
    keep = [_field(phi, p.nx * p.ny) for phi, p in zip(phis, params)]
    ptrs = (_DP * n)(*[_dp(a) for a in keep])
    h = _VP()
    rc = load().clb_batch_init(ctypes.byref(h), n, P, ptrs, B, _VP(stream) if stream else None)
    _bcheck(rc, None)
    return h.value


def clb_batch_step(b, n: int):
    _bcheck(load().clb_batch_step(b, int(n)), b)


def clb_batch_set_active(b, active):
    a = (ctypes.c_int32 * len(active))(*[int(bool(v)) for v in active])
    _bcheck(load().clb_batch_set_active(b, a), b)


def clb_batch_set_tiling(b, choice: int):
    _bcheck(load().clb_batch_set_tiling(b, int(choice)), b)


def clb_batch_set_mode(b, mode: int):
    _bcheck(load().clb_batch_set_mode(b, int(mode)), b)


def clb_batch_barrier_selftest(b, limit_cycles: int):
    """Returns the library's status (CLB_ERR_TIMEOUT expected); see clb.h."""
    return int(load().clb_batch_barrier_selftest(b, int(limit_cycles)))


def clb_batch_tune(b, steps: int = 4) -> int:
    ch = ctypes.c_int32(-1)
    _bcheck(load().clb_batch_tune(b, int(steps), ctypes.byref(ch)), b)
    return ch.value


def clb_batch_nusselt(b, ncase: int, side: int = W) -> np.ndarray:
    out = np.zeros(ncase)
    _bcheck(load().clb_batch_nusselt(b, int(side), _dp(out)), b)
    return out


def clb_batch_macros(b, c: int, nx: int, ny: int):
    out = [np.empty((ny, nx)) for _ in range(4)]
    _bcheck(load().clb_batch_macros(b, int(c), *[_dp(a) for a in out]), b)
    return tuple(out)


def clb_batch_nodes(b) -> int:
    return int(load().clb_batch_nodes(b))


def clb_batch_time(b) -> int:
    return int(load().clb_batch_time(b))


def clb_batch_sync(b):
    _bcheck(load().clb_batch_sync(b), b)


def clb_batch_destroy(b):
    if b:
        load().clb_batch_destroy(b)


class Batch:
    """Owns one batch handle; cases are indexed 0..n-1."""

    def __init__(self, params, phis, bcs, stream=None):
        self.params = list(params)
        self.handle = clb_batch_init(self.params, phis, bcs, stream)

    def __len__(self):
        return len(self.params)

    def step(self, n: int):
        clb_batch_step(self.handle, n)

    def set_active(self, active):
        clb_batch_set_active(self.handle, active)

    def tune(self, steps: int = 4) -> int:
        return clb_batch_tune(self.handle, steps)

    def set_tiling(self, choice: int):
        clb_batch_set_tiling(self.handle, choice)

    def set_mode(self, mode: int):
        clb_batch_set_mode(self.handle, mode)

    def barrier_selftest(self, limit_cycles: int) -> int:
        return clb_batch_barrier_selftest(self.handle, limit_cycles)

    def nusselt(self, side: int = W) -> np.ndarray:
        return clb_batch_nusselt(self.handle, len(self), side)

    def macros(self, c: int):
        p = self.params[c]
        return clb_batch_macros(self.handle, c, p.nx, p.ny)

    @property
    def nodes(self) -> int:
        return clb_batch_nodes(self.handle)

    @property
    def time(self) -> int:
        return clb_batch_time(self.handle)

    def sync(self):
        clb_batch_sync(self.handle)

    def close(self):
        if self.handle:
            clb_batch_destroy(self.handle)
            self.handle = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
