"""Matched set-ups for the oracle and the CUDA path (test glue only).

Both sides receive the same physical description and the same seeded
arrays; each maps it to lattice parameters on its own."""
from __future__ import annotations

import numpy as np

import oracle
from paper_2110_05943_gb300 import clb

CAVITY = ("wall", "wall", "wall", "wall")
CHANNEL_X = ("periodic", "periodic", "wall", "wall")
PERIODIC = ("periodic",) * 4


def build(nx, ny, phi, Ra=1e4, Da=1e-2, Pr=1.0, sigma=1.0, J=1.0, Gamma=1.0, L=None, nu=None,
          ax=0.0, ay=0.0, forchheimer=True, shift=True, T0=0.5, T_init=0.5, dT=1.0, precision=0,
          kind=CAVITY, u=(0.0,) * 4, v=(0.0,) * 4, T=(1.0, 0.0, None, None), ay_row=None,
          nthreads=None, stream=None, with_oracle=True):
    """Returns (oracle.Oracle or None, clb.Simulation)."""
    phi_arr = np.ascontiguousarray(np.broadcast_to(np.asarray(phi, dtype=np.float64), (ny, nx)))
    orc = None
    if with_oracle:
        p = oracle.Problem(nx=nx, ny=ny, Ra=Ra, Da=Da, Pr=Pr, J=J, Gamma=Gamma, sigma=sigma, L=L, nu=nu,
                           dT=dT, T0=T0, T_init=T_init, ax=ax, ay=ay, forchheimer=forchheimer, shift=shift,
                           walls=oracle.Walls(kind, u, v, T))
        orc = oracle.Oracle(p, phi=phi_arr, ay_row=ay_row, nthreads=nthreads)
    cp = clb.clb_params_default(nx=nx, ny=ny, Ra=Ra, Da=Da, Pr=Pr, J=J, Gamma=Gamma, sigma=sigma,
                                L=0.0 if L is None else L, nu=0.0 if nu is None else nu, dT=dT, T0=T0,
                                T_init=T_init, ax=ax, ay=ay, forchheimer=int(forchheimer), shift=int(shift),
                                precision=precision)
    bc = clb.clb_bc(kind, u, v, T)
    sim = clb.Simulation.create(cp, phi_arr, bc, ay_row=ay_row, stream=stream)
    return orc, sim


def rel_err(a, b) -> float:
    """max_x |a - b| / max_x |b| (the parity metric; b is the oracle)."""
    den = float(np.max(np.abs(b)))
    num = float(np.max(np.abs(a - b)))
    return num / den if den > 0 else num


# Smallest field scales the relative error is taken against: density
# deviations below 1e-4 and speeds below 1e-6 (3 % of the Ma^2 ~ 3e-3
# density variation of a developed cavity flow, 2e-5 of u_c = 0.058).  Below
# them the rounding of rho ~ 1 accumulated over a few hundred steps
# (~3e-15) already reads as 1e-10 of the field maximum -- e.g. the first
# steps of a 4096^2 cavity.
FLOORS = {"rho-1": 1e-4, "ux": 1e-6, "uy": 1e-6, "T": 0.0}


def field_errors(gpu, orc_fields):
    """Per-field parity errors max|a - b| / max(max|b|, floor); density
    compared as rho - 1."""
    names = ("rho-1", "ux", "uy", "T")
    out = {}
    for k, (a, b) in enumerate(zip(gpu, orc_fields)):
        if k == 0:
            a, b = a - 1.0, b - 1.0
        den = max(float(np.max(np.abs(b))), FLOORS[names[k]])
        out[names[k]] = float(np.max(np.abs(a - b))) / den if den > 0 else float(np.max(np.abs(a - b)))
    return out
