"""Explicit upwind saturation update for piecewise-constant saturation.

Definition 3 (Eq. saturationDG) with k = 0: the volume term vanishes for
constant test functions and the saturation penalty term is dropped (reading
R10, finite-volume form), which leaves, for every cell e,

  phi_e |e| (s_e^{n+1} - s_e^n) / dt = - sum_{f in de} F_f^{out,e} f_w(chi_f(s^n))

with chi of Eq. upwind: on an interior face the value of the cell the flux
leaves (s|e1 when u.n >= 0 with n from e1 to e2, else s|e2); on a boundary
face the cell value when the flux leaves the domain and the prescribed
inflow saturation s_D when it enters (reading R11).

Time step (reading R12): dt = cfl * min_e phi_e |e| / (L_f * sum_f max(F_f^{out,e}, 0))
over cells with positive outflow, L_f = max f_w'; an optional dt_max caps it.
"""
from __future__ import annotations

import numpy as np

from .grid import Grid
from .physics import frac_flow


def cfl_dt(grid: Grid, F: np.ndarray, poro: np.ndarray, Lf: float, cfl: float,
           dt_max: float = np.inf) -> float:
    outpos = np.zeros(grid.n_cells)
    f = grid.interior
    np.add.at(outpos, grid.fe1[f], np.maximum(F[f], 0.0))
    np.add.at(outpos, grid.fe2[f], np.maximum(-F[f], 0.0))
    np.add.at(outpos, grid.bcell, np.maximum(F[grid.bface] * grid.bsign, 0.0))
    m = outpos > 0.0
    if not np.any(m):
        return float(dt_max)
    dt = cfl * np.min(poro[m] * grid.vol / (Lf * outpos[m]))
    return float(min(dt, dt_max))


def fv_update(grid: Grid, s: np.ndarray, F: np.ndarray, poro: np.ndarray, dt: float,
              s_D: np.ndarray, eta_w: float, eta_o: float, law: str):
    """One explicit Euler step. Returns (s_new, boundary_outflow) where
    boundary_outflow = sum over boundary faces of F^out f_w(chi), so that the
    total water volume changes by exactly -dt * boundary_outflow."""
    fw = lambda x: frac_flow(x, eta_w, eta_o, law)  # noqa: E731
    net = np.zeros(grid.n_cells)
    f = grid.interior
    e1, e2 = grid.fe1[f], grid.fe2[f]
    s_up = np.where(F[f] >= 0.0, s[e1], s[e2])
    G = F[f] * fw(s_up)
    np.add.at(net, e1, G)
    np.add.at(net, e2, -G)
    Fout = F[grid.bface] * grid.bsign
    s_upb = np.where(Fout >= 0.0, s[grid.bcell], s_D)
    Gb = Fout * fw(s_upb)
    np.add.at(net, grid.bcell, Gb)
    s_new = s - dt / (poro * grid.vol) * net
    return s_new, float(np.sum(Gb))
