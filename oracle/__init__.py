"""FP64 CPU oracle for the REV-scale cascaded lattice Boltzmann method
(Feng, Liu & He, arXiv:2110.05943).

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  It shares no code with ``paper_2110_05943_gb300`` and never imports
it.  The heavy lifting is the plain C file ``clb_oracle.c`` next to this one
(literal dense matrix products, no FMA contraction); this module builds it
with gcc, maps the dimensionless groups of Sec. 3 to lattice parameters and
adds the post-processing of Sec. 3 (Nusselt number, residuals, error norms).

Parameter mapping (written from the paper):
  * Eq. 46: 1/s_v = 1/2 + Ma J L sqrt(3 Pr) / sqrt(Ra) and
            1/zeta_a = 1/2 + Gamma c_s^2 (1/s_v - 1/2) / (J c_sT^2 Pr),
    with Ma = 0.1 and c = dt = 1 (Sec. 3.2);
  * channel flows (Sec. 3.1) fix the viscosity instead:
            1/s_v = 1/2 + J nu / c_s^2 (nu = H u_1 / Re in the paper);
  * Eq. 38: K = Da L^2, g beta = Ra nu alpha / (Delta T L^3), alpha = nu / Pr;
  * Eq. 15 text: nu_e = c_s^2 (1/s_v - 1/2); Eq. 37: alpha_e = c_sT^2 (1/zeta_a - 1/2);
  * Sec. 3 constants: s_0 = s_1 = 1, s_b = s_v, s_3 = 1.2, s_4 = 1.8,
    zeta_T = zeta_e = zeta_nu = 1, varpi = 1/4 (c_sT^2 = 1/8), J = 1.
  * Bulk rate: with s_3 = 1.2 and s_4 = 1.8 the linearised scheme is stable
    only for s_b >= 1.19, so s_b = s_v is kept where s_v >= 1.2 and raised
    to 1.2 below that (Eq. 46 gives s_v < 1.2 for the Ra = 1e3 rows of
    Table 1 and for large grids).  s_b sets only the bulk viscosity, which
    does not appear in the incompressible equations (Eqs. 1-3).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "clb_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liborc.so")
_lock = threading.Lock()
_lib = None

CS2 = 1.0 / 3.0  # D2Q9 sound speed squared, c_s = c / sqrt(3) (Eq. 15 text)

W, E, S, N = 0, 1, 2, 3


def build(force: bool = False) -> str:
    """Compile clb_oracle.c into _build/liborc.so (plain gcc, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-std=c11",
           "-shared", "-fPIC", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Cfg(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int),
        ("kind", ctypes.c_int * 4),
        ("uw", ctypes.c_double * 4), ("vw", ctypes.c_double * 4),
        ("tdir", ctypes.c_int * 4),
        ("Tw", ctypes.c_double * 4),
        ("nu", ctypes.c_double), ("nu_e", ctypes.c_double), ("K", ctypes.c_double),
        ("gbeta", ctypes.c_double),
        ("sigma", ctypes.c_double), ("varpi", ctypes.c_double), ("T0", ctypes.c_double),
        ("ax", ctypes.c_double),
        ("s0", ctypes.c_double), ("s1", ctypes.c_double), ("sb", ctypes.c_double),
        ("sv", ctypes.c_double), ("s3", ctypes.c_double), ("s4", ctypes.c_double),
        ("zT", ctypes.c_double), ("za", ctypes.c_double), ("ze", ctypes.c_double),
        ("zn", ctypes.c_double),
        ("forchheimer", ctypes.c_int), ("shift", ctypes.c_int),
        ("nthreads", ctypes.c_int),
    ]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            dp = ctypes.POINTER(ctypes.c_double)
            d = ctypes.c_double
            L.orc_create.restype = ctypes.c_void_p
            L.orc_create.argtypes = [ctypes.POINTER(_Cfg), dp, dp]
            L.orc_destroy.argtypes = [ctypes.c_void_p]
            L.orc_step.argtypes = [ctypes.c_void_p, ctypes.c_int64]
            L.orc_macros.argtypes = [ctypes.c_void_p, dp, dp, dp, dp]
            L.orc_set_fields.argtypes = [ctypes.c_void_p, dp, dp, dp, dp]
            L.orc_get_state.argtypes = [ctypes.c_void_p, dp, dp]
            L.orc_set_state.argtypes = [ctypes.c_void_p, dp, dp]
            L.orc_matrix_M.argtypes = [dp]
            L.orc_matrix_MT.argtypes = [dp]
            L.orc_matrix_N.argtypes = [d, d, d, dp]
            L.orc_matrix_Ninv.argtypes = [d, d, d, dp]
            L.orc_matrix_NT.argtypes = [d, d, d, dp]
            L.orc_matrix_NTinv.argtypes = [d, d, d, dp]
            L.orc_matrix_Lambda.argtypes = [d, d, d, d, d, d, dp]
            L.orc_invert.argtypes = [ctypes.c_int, dp, dp]
            L.orc_invert.restype = ctypes.c_int
            L.orc_meq_central.argtypes = [d, dp]
            L.orc_S_central.argtypes = [d, d, d, dp]
            L.orc_meq_raw.argtypes = [d, d, d, d, dp]
            L.orc_S_raw.argtypes = [d, d, d, d, d, d, dp]
            L.orc_neq_central.argtypes = [d, d, d, dp]
            L.orc_neq_raw.argtypes = [d, d, d, d, d, dp]
            L.orc_ergun_Fphi.argtypes = [d]
            L.orc_ergun_Fphi.restype = d
            L.orc_feq.argtypes = [d, d, d, d, dp]
            L.orc_geq.argtypes = [d, d, d, d, d, dp]
            L.orc_collide_flow.argtypes = [dp, d, d, d, d, d, d, d, d, d, d, d, d, ctypes.c_int, dp]
            L.orc_collide_thermal.argtypes = [dp, d, d, d, d, d, d, d, d, d, ctypes.c_int, dp]
            L.orc_point_velocity.argtypes = [ctypes.POINTER(_Cfg), d, d, d, d, d, d, dp]
            L.orc_sizeof_cfg.restype = ctypes.c_int
            assert L.orc_sizeof_cfg() == ctypes.sizeof(_Cfg), "orc_cfg layout mismatch"
            _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


# ------------------------------------------------------------ small wrappers
def mat(name: str, *args) -> np.ndarray:
    """Return one of the oracle's matrices as a numpy array."""
    n = 5 if name in ("MT", "NT", "NTinv") else 9
    out = np.zeros(n * n)
    getattr(lib(), "orc_matrix_" + name)(*[float(a) for a in args], _p(out))
    return out.reshape(n, n)


def vec(name: str, n: int, *args) -> np.ndarray:
    out = np.zeros(n)
    getattr(lib(), "orc_" + name)(*[float(a) for a in args], _p(out))
    return out


def invert(A: np.ndarray) -> np.ndarray:
    A = np.ascontiguousarray(A, dtype=np.float64)
    out = np.zeros_like(A)
    rc = lib().orc_invert(A.shape[0], _p(A), _p(out))
    if rc != 0:
        raise np.linalg.LinAlgError("singular")
    return out


def ergun_Fphi(phi: float) -> float:
    return lib().orc_ergun_Fphi(float(phi))


def feq(rho, ux, uy, phi) -> np.ndarray:
    return vec("feq", 9, rho, ux, uy, phi)


def geq(T, ux, uy, sigma, varpi=0.25) -> np.ndarray:
    return vec("geq", 5, T, ux, uy, sigma, varpi)


def collide_flow(f, rho, ux, uy, Fx, Fy, phi, sv, s3=1.2, s4=1.8, s0=1.0, s1=1.0, sb=None,
                 shift=True) -> np.ndarray:
    f = np.ascontiguousarray(f, dtype=np.float64)
    out = np.zeros(9)
    sb = sv if sb is None else sb
    lib().orc_collide_flow(_p(f), rho, ux, uy, Fx, Fy, phi, s0, s1, sb, sv, s3, s4, int(shift), _p(out))
    return out


def collide_thermal(g, T, ux, uy, sigma, za, varpi=0.25, zT=1.0, ze=1.0, zn=1.0,
                    shift=True) -> np.ndarray:
    g = np.ascontiguousarray(g, dtype=np.float64)
    out = np.zeros(5)
    lib().orc_collide_thermal(_p(g), T, ux, uy, sigma, varpi, zT, za, ze, zn, int(shift), _p(out))
    return out


# ------------------------------------------------------------ configuration
@dataclass
class Walls:
    """Boundary specification, sides ordered W, E, S, N.

    kind: 'periodic' or 'wall' per side (W/E and S/N must agree on periodicity);
    u, v: wall velocity; T: wall temperature or None for an adiabatic wall."""
    kind: tuple = ("wall", "wall", "wall", "wall")
    u: tuple = (0.0, 0.0, 0.0, 0.0)
    v: tuple = (0.0, 0.0, 0.0, 0.0)
    T: tuple = (1.0, 0.0, None, None)


def cavity_walls(Th=1.0, Tc=0.0) -> Walls:
    """Sec. 3.2: hot left wall, cold right wall, adiabatic top and bottom, no slip."""
    return Walls(("wall",) * 4, (0.0,) * 4, (0.0,) * 4, (Th, Tc, None, None))


@dataclass
class Problem:
    nx: int
    ny: int
    Ra: float
    Da: float
    Pr: float = 1.0
    J: float = 1.0
    Gamma: float = 1.0
    sigma: float = 1.0
    Ma: float = 0.1
    L: float | None = None          # characteristic length; default ny - 1
    nu: float | None = None         # fix the fluid viscosity (channel flows)
    dT: float = 1.0
    T0: float = 0.5
    T_init: float = 0.5
    ax: float = 0.0
    ay: float = 0.0
    forchheimer: bool = True
    shift: bool = True
    varpi: float = 0.25
    s3: float = 1.2
    s4: float = 1.8
    sb: float | None = None         # bulk rate; None: s_v, raised to SB_STABLE when s_v < SB_STABLE
    walls: Walls = field(default_factory=cavity_walls)


# Smallest bulk relaxation rate for which the printed rate set s_3 = 1.2,
# s_4 = 1.8 (Sec. 3) is linearly stable (von Neumann analysis of the
# linearised step, tests/test_oracle_stability.py: threshold 1.19).
SB_STABLE = 1.2


@dataclass
class Lattice:
    sb: float
    sv: float
    za: float
    nu: float
    nu_e: float
    alpha: float
    alpha_e: float
    K: float
    gbeta: float
    L: float


def lattice_params(p: Problem) -> Lattice:
    """Dimensionless groups -> lattice parameters (Eqs. 38, 46; Sec. 3.1)."""
    L = float(p.ny - 1) if p.L is None else float(p.L)
    if p.nu is None:
        if p.Ra <= 0:
            raise ValueError("Ra must be positive when the viscosity is not given")
        inv_sv = 0.5 + p.Ma * p.J * L * math.sqrt(3.0 * p.Pr) / math.sqrt(p.Ra)   # Eq. 46
    else:
        inv_sv = 0.5 + p.J * p.nu / CS2
    nu_e = CS2 * (inv_sv - 0.5)
    nu = nu_e / p.J
    cT2 = 0.5 * p.varpi
    inv_za = 0.5 + p.Gamma * CS2 * (inv_sv - 0.5) / (p.J * cT2 * p.Pr)           # Eq. 46
    alpha = nu / p.Pr
    alpha_e = cT2 * (inv_za - 0.5)                                             # Eq. 37
    K = p.Da * L * L                                                           # Eq. 38
    gbeta = p.Ra * nu * alpha / (p.dT * L ** 3)                                # Eq. 38
    sv = 1.0 / inv_sv
    sb = p.sb if p.sb is not None else max(sv, SB_STABLE)
    return Lattice(sb=sb, sv=sv, za=1.0 / inv_za, nu=nu, nu_e=nu_e, alpha=alpha,
                   alpha_e=alpha_e, K=K, gbeta=gbeta, L=L)


def _cfg(p: Problem, nthreads: int) -> _Cfg:
    lat = lattice_params(p)
    w = p.walls
    kinds = [1 if k == "wall" else 0 for k in w.kind]
    if kinds[0] != kinds[1] or kinds[2] != kinds[3]:
        raise ValueError("opposite sides must agree on periodicity")
    if (kinds[0] and p.nx < 4) or (kinds[2] and p.ny < 4):
        raise ValueError("a walled direction needs at least 4 nodes")
    c = _Cfg()
    c.nx, c.ny = p.nx, p.ny
    for s in range(4):
        c.kind[s] = kinds[s]
        c.uw[s] = float(w.u[s])
        c.vw[s] = float(w.v[s])
        c.tdir[s] = 0 if w.T[s] is None else 1
        c.Tw[s] = 0.0 if w.T[s] is None else float(w.T[s])
    c.nu, c.nu_e, c.K, c.gbeta = lat.nu, lat.nu_e, lat.K, lat.gbeta
    c.sigma, c.varpi, c.T0, c.ax = p.sigma, p.varpi, p.T0, p.ax
    c.s0, c.s1, c.sb, c.sv, c.s3, c.s4 = 1.0, 1.0, lat.sb, lat.sv, p.s3, p.s4
    c.zT, c.za, c.ze, c.zn = 1.0, lat.za, 1.0, 1.0
    c.forchheimer = int(bool(p.forchheimer))
    c.shift = int(bool(p.shift))
    c.nthreads = int(nthreads)
    return c


def default_threads() -> int:
    return max(1, len(os.sched_getaffinity(0)))


class Oracle:
    """One simulation on the CPU.  Fields are (ny, nx) row-major, x fastest."""

    def __init__(self, p: Problem, phi=None, ay_row=None, nthreads: int | None = None):
        self.p = p
        self.lat = lattice_params(p)
        self.nthreads = default_threads() if nthreads is None else nthreads
        self.cfg = _cfg(p, self.nthreads)
        phi = np.full((p.ny, p.nx), 1.0) if phi is None else phi
        if np.isscalar(phi):
            phi = np.full((p.ny, p.nx), float(phi))
        self.phi = np.ascontiguousarray(phi, dtype=np.float64).reshape(p.ny, p.nx)
        ay = np.full(p.ny, float(p.ay)) if ay_row is None else np.asarray(ay_row, dtype=np.float64)
        self.ay = np.ascontiguousarray(ay).reshape(p.ny)
        self.h = lib().orc_create(ctypes.byref(self.cfg), _p(self.phi), _p(self.ay))
        if not self.h:
            raise MemoryError("orc_create failed")
        self.steps = 0
        n = p.nx * p.ny
        self.set_fields(np.ones(n), np.zeros(n), np.zeros(n), np.full(n, p.T_init))

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            lib().orc_destroy(h)
            self.h = None

    def set_fields(self, rho, ux, uy, T):
        arrs = [np.ascontiguousarray(np.broadcast_to(a, (self.p.ny * self.p.nx,)), dtype=np.float64)
                for a in (rho, ux, uy, T)]
        lib().orc_set_fields(self.h, *[_p(a) for a in arrs])
        self.steps = 0

    def step(self, n: int):
        lib().orc_step(self.h, int(n))
        self.steps += int(n)

    def macros(self):
        ny, nx = self.p.ny, self.p.nx
        out = [np.zeros((ny, nx)) for _ in range(4)]
        lib().orc_macros(self.h, *[_p(a) for a in out])
        return tuple(out)  # rho, ux, uy, T

    def state(self):
        n = self.p.nx * self.p.ny
        f, g = np.zeros(9 * n), np.zeros(5 * n)
        lib().orc_get_state(self.h, _p(f), _p(g))
        return f.reshape(self.p.ny, self.p.nx, 9), g.reshape(self.p.ny, self.p.nx, 5)

    def set_state(self, f, g):
        f = np.ascontiguousarray(f, dtype=np.float64)
        g = np.ascontiguousarray(g, dtype=np.float64)
        lib().orc_set_state(self.h, _p(f), _p(g))

    def nusselt(self, side: int = W) -> float:
        _, _, _, T = self.macros()
        return nusselt(T, side, self.lat.L, self.p.dT)


# ------------------------------------------------------------ post-processing
def nusselt(T: np.ndarray, side: int, L: float, dT: float = 1.0) -> float:
    """Mean Nusselt number of Sec. 3.2: Nu(y) = -L dT/dx|wall / Delta T,
    averaged over the wall by the trapezoid rule (nodes on the wall, spacing 1).
    The wall-normal derivative is the one-sided second-order difference
    (-3 T_0 + 4 T_1 - T_2)/2 taken into the domain; for the W/S walls this is
    dT/dn with n along +x/+y, for the E/N walls the sign flips so that the
    same formula -L dT/dx (or dT/dy) is reported."""
    T = np.asarray(T, dtype=np.float64)
    if side == W:
        d = (-3.0 * T[:, 0] + 4.0 * T[:, 1] - T[:, 2]) / 2.0
    elif side == E:
        d = (3.0 * T[:, -1] - 4.0 * T[:, -2] + T[:, -3]) / 2.0
    elif side == S:
        d = (-3.0 * T[0, :] + 4.0 * T[1, :] - T[2, :]) / 2.0
    else:
        d = (3.0 * T[-1, :] - 4.0 * T[-2, :] + T[-3, :]) / 2.0
    nu_local = -L * d / dT
    n = nu_local.size
    return float((nu_local[0] * 0.5 + nu_local[1:-1].sum() + nu_local[-1] * 0.5) / (n - 1))


def residual(a_now: np.ndarray, a_prev: np.ndarray) -> float:
    """||a^n - a^(n-k)||_2 / ||a^n||_2 over the whole field."""
    den = math.sqrt(float(np.sum(a_now * a_now)))
    num = math.sqrt(float(np.sum((a_now - a_prev) ** 2)))
    return num / den if den > 0 else num


def global_error(exact: np.ndarray, numeric: np.ndarray) -> float:
    """Relative global error of Eq. 45."""
    return math.sqrt(float(np.sum((exact - numeric) ** 2))) / math.sqrt(float(np.sum(exact ** 2)))
