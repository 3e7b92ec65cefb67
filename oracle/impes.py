"""High-dimensional two-phase scheme (Algorithm 1) with piecewise-constant
saturation (no limiter is needed for k = 0).

Per step n: (a) pressure of Definition 1 with the mobilities of s^n,
(b) velocity of Definition 2 from that pressure, (c) saturation of
Definition 3, with the time step of ``transport.cfl_dt``. The initial
projection of s0 onto piecewise constants is the cell average, so a per-cell
s0 is used as given.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.sparse.linalg as spla

from .grid import Grid
from .physics import total_mobility, max_frac_flow_slope
from .swip import pressure_system, default_penalty_scale
from .transport import cfl_dt, fv_update
from .velocity import face_fluxes


@dataclass
class FineModel:
    grid: Grid
    perm: np.ndarray
    poro: np.ndarray
    eta_w: float
    eta_o: float
    law: str
    bc_type: np.ndarray
    p_D: np.ndarray
    v_N: np.ndarray
    s_D: np.ndarray
    c_pen: float
    cfl: float = 0.5
    dt_max: float = np.inf
    dt_fixed: float | None = None
    swapped: bool = False

    def __post_init__(self):
        self.Lf = max_frac_flow_slope(self.eta_w, self.eta_o, self.law)

    @classmethod
    def from_problem(cls, prob, c_pen=None, **kw):
        g = Grid(prob.nx, prob.ny, prob.Lx, prob.Ly)
        if c_pen is None:
            c_pen = default_penalty_scale(prob.eta_w, prob.eta_o)
        return cls(grid=g, perm=prob.perm, poro=prob.poro, eta_w=prob.eta_w,
                   eta_o=prob.eta_o, law=prob.relperm, bc_type=prob.bc_type,
                   p_D=prob.p_D, v_N=prob.v_N, s_D=prob.s_D, c_pen=c_pen,
                   cfl=prob.cfl, **kw)

    def mobility(self, s):
        return total_mobility(s, self.eta_w, self.eta_o, self.law)

    def solve_pressure(self, gamma, source=None):
        K, l = pressure_system(self.grid, self.perm, gamma, self.c_pen, self.bc_type,
                               self.p_D, self.v_N, swapped=self.swapped, source=source)
        return spla.spsolve(K.tocsc(), l)

    def fluxes(self, p, gamma):
        return face_fluxes(self.grid, self.perm, gamma, self.c_pen, self.bc_type,
                           self.p_D, self.v_N, p, swapped=self.swapped)

    def time_step(self, F):
        if self.dt_fixed is not None:
            return float(self.dt_fixed)
        return cfl_dt(self.grid, F, self.poro, self.Lf, self.cfl, self.dt_max)

    def step(self, s):
        lam = self.mobility(s)
        p = self.solve_pressure(lam)
        F = self.fluxes(p, lam)
        dt = self.time_step(F)
        s_new, bout = fv_update(self.grid, s, F, self.poro, dt, self.s_D,
                                self.eta_w, self.eta_o, self.law)
        return dict(p=p, F=F, dt=dt, s=s_new, boundary_outflow=bout)

    def run(self, s0, n_steps):
        s = np.array(s0, dtype=np.float64)
        hist = []
        for _ in range(n_steps):
            r = self.step(s)
            s = r["s"]
            hist.append(r)
        return s, hist
