"""Piecewise-linear DG saturation step (Definition 3, Eq. saturationDG, with
k = 1) and the mass-conservative slope limiter (Section 3.4, Eq.
limiterMain), FP64 on the CPU. Test infrastructure: only tests, the smoke
check and the benchmark's CPU leg use this module.

State: per cell e the coefficients c = (c0, c1, c2) of
    s_h|e = c0 + c1 psi1 + c2 psi2,  psi1 = 2 (x - xc)/hx,  psi2 = 2 (y - yc)/hy,
the pressure's local basis (reading R5); c0 is the cell mean. In reference
coordinates r, t in [-1, 1] of the cell, psi1 = r and psi2 = t.

Velocity: the lowest-order Raviart-Thomas field of the face fluxes F of
Definition 2 (F = int_f u.n with n along +x / +y): in a cell with left,
right, bottom and top fluxes F_l, F_r, F_b, F_t,
    u_x = (F_l (1 - r) + F_r (1 + r)) / (2 hy),  u_y = (F_b (1 - t) + F_t (1 + t)) / (2 hx).

Step (explicit Euler, gravity and sources zero): for the basis functions
psi_j with L2(e) norms |e| m_j, m = (1, 1/3, 1/3),
    phi_e |e| m_j (c_j^{n+1} - c_j^n) / dt = R_j,
    R_j = int_e f(s) u . grad psi_j dx - sum_{f in de} int_f (u . n_out) f(s_up) psi_j ds,
with s_up the trace of the cell the flux leaves (Eq. upwind; F >= 0 takes the
first cell, reading R11) and s_D on inflow boundary faces.
Readings where the paper leaves the choice open:
  - quadrature: 3 x 3 Gauss-Legendre points in the cell, 3 on a face (f_w is
    rational, so no rule is exact; the rule integrates the linear-flux case
    exactly);
  - the saturation penalty term of Eq. saturationDG is dropped, as for k = 0
    (reading R10): with the pressure's penalty sigma_f it would bound the
    explicit step far below the advective CFL bound in these units, and the
    upwind flux with the limiter provides the stabilisation;
  - the time step is the CFL step of the finite-volume scheme divided by
    2k + 1 = 3;
  - the pressure and the fluxes take the mobilities at the cell means.

Limiter (applied to s^{n+1} with the velocity of the step, Algorithm 1 step
2(d)): the shock detector
    eta(e) = sum over the upstream faces f of e (u . n_out < 0) of
             |int_f [s] ds| / (0.08 d sqrt(h_e) |e|),  d = 2, h_e = diam(e),
with [s] the difference of the traces (s_D on an inflow boundary face); a
cell is flagged if eta(e) > 1 or s_h leaves [0, 1] in e (at a vertex, as
s_h is linear). For a flagged cell and each face neighbour i,
g_i = grad s . (b_i - b_e) and d_i = mean_i - mean_e give m_i by the three
cases of Section 3.4, and the limited function keeps the cell mean with the
slope scaled by min_i m_i. (Reading: the printed Eq. limiterMain adds the
scaled gradient term to s itself, which would double the slope where
m_i = 1; the cell mean plus the scaled linear part is the reading that
leaves unflagged-like cells unchanged and conserves the mean.) The
detector's jump is taken in absolute value (reading).
"""
from __future__ import annotations

import numpy as np

from .grid import Grid
from .physics import frac_flow
from .transport import cfl_dt

GAUSS3_X = np.array([-np.sqrt(0.6), 0.0, np.sqrt(0.6)])
GAUSS3_W = np.array([5.0 / 9.0, 8.0 / 9.0, 5.0 / 9.0])
MASS = np.array([1.0, 1.0 / 3.0, 1.0 / 3.0])


def dg_time_step(grid: Grid, F: np.ndarray, poro: np.ndarray, Lf: float, cfl: float,
                 dt_max: float = np.inf) -> float:
    """CFL step of the finite-volume scheme (reading R12) divided by 2k + 1 = 3."""
    return cfl_dt(grid, F, poro, Lf, cfl, dt_max * 3.0) / 3.0


def _cell_faces(grid: Grid):
    """Left, right, bottom and top face of every cell."""
    j, i = grid.cj, grid.ci
    fl = j * (grid.nx + 1) + i
    fb = grid.nxf + j * grid.nx + i
    return fl, fl + 1, fb, fb + grid.nx


def _neighbour(grid: Grid, side: int):
    """Cell across the left (0), right (1), bottom (2) or top (3) face, or -1."""
    i, j, nx, ny = grid.ci, grid.cj, grid.nx, grid.ny
    e = np.arange(grid.n_cells)
    if side == 0:
        return np.where(i > 0, e - 1, -1)
    if side == 1:
        return np.where(i < nx - 1, e + 1, -1)
    if side == 2:
        return np.where(j > 0, e - nx, -1)
    return np.where(j < ny - 1, e + nx, -1)


def _boundary_index(grid: Grid, side: int):
    """Boundary face index (left side, right side, bottom side, top side
    numbering) of each cell's face on `side`, for cells on that side."""
    i, j, nx, ny = grid.ci, grid.cj, grid.nx, grid.ny
    return [j, ny + j, 2 * ny + i, 2 * ny + nx + i][side]


# points of a face in reference coordinates (r, t) and the face's outward sign
_SIDES = [(-1.0, None, -1.0), (1.0, None, 1.0), (None, -1.0, -1.0), (None, 1.0, 1.0)]


def _trace(c: np.ndarray, side: int, q: np.ndarray) -> np.ndarray:
    """s_h at the face points q (tangential coordinate) of the cells' face `side`."""
    r, t, _ = _SIDES[side]
    if r is not None:
        return c[:, 0, None] + c[:, 1, None] * r + c[:, 2, None] * q[None, :]
    return c[:, 0, None] + c[:, 1, None] * q[None, :] + c[:, 2, None] * t


def dg_step(grid: Grid, c: np.ndarray, F: np.ndarray, poro: np.ndarray, dt: float,
            s_D: np.ndarray, eta_w: float, eta_o: float, law: str):
    """One explicit Euler step of Definition 3 with k = 1 (module docstring).
    c: (n_cells, 3). Returns (c_new, boundary_outflow) with boundary_outflow
    = sum over boundary faces of the outward flux times the face mean of
    f(s_up), so that sum_e phi_e |e| c0_e changes by exactly -dt times it."""
    fw = lambda s: frac_flow(s, eta_w, eta_o, law)  # noqa: E731
    hx, hy = grid.hx, grid.hy
    fl, fr, fb, ft = _cell_faces(grid)
    Fl, Fr, Fb, Ft = F[fl], F[fr], F[fb], F[ft]
    R = np.zeros((grid.n_cells, 3))
    # volume term: f(s) u . grad psi_j, grad psi1 = (2/hx, 0), grad psi2 = (0, 2/hy)
    for a, ra in enumerate(GAUSS3_X):
        ux = (Fl * (1.0 - ra) + Fr * (1.0 + ra)) / (2.0 * hy)
        for b, tb in enumerate(GAUSS3_X):
            uy = (Fb * (1.0 - tb) + Ft * (1.0 + tb)) / (2.0 * hx)
            w = GAUSS3_W[a] * GAUSS3_W[b] * grid.vol / 4.0
            f = fw(c[:, 0] + c[:, 1] * ra + c[:, 2] * tb)
            R[:, 1] += w * f * ux * (2.0 / hx)
            R[:, 2] += w * f * uy * (2.0 / hy)
    # face terms: -int_f (u . n_out) f(s_up) psi_j ds for the four faces of each cell
    bout = 0.0
    for side, Fs in enumerate((Fl, Fr, Fb, Ft)):
        r, t, sgn = _SIDES[side]
        Fout = sgn * Fs  # outward flux of the cell through this face
        own = _trace(c, side, GAUSS3_X)
        nb = _neighbour(grid, side)
        inside = nb >= 0
        up = own.copy()
        if np.any(inside):
            # the neighbour's trace on the same face: its opposite side
            other = _trace(c[nb[inside]], side ^ 1, GAUSS3_X)
            up[inside] = np.where(Fout[inside, None] >= 0.0, own[inside], other) if sgn > 0 else \
                np.where(Fout[inside, None] > 0.0, own[inside], other)
        bnd = ~inside
        if np.any(bnd):
            sD = s_D[_boundary_index(grid, side)[bnd]]
            up[bnd] = np.where(Fout[bnd, None] >= 0.0, own[bnd], sD[:, None])
        g = fw(up)  # (n_cells, 3 points)
        ln = hy if r is not None else hx
        # psi_j at the face points
        if r is not None:
            psi = np.stack([np.ones(3), np.full(3, r), GAUSS3_X])
        else:
            psi = np.stack([np.ones(3), GAUSS3_X, np.full(3, t)])
        # int_f (u.n) f psi_j ds = Fout / |f| * sum_q w_q (|f|/2) g_q psi_j(q)
        R -= (Fout[:, None] * 0.5) * (g * GAUSS3_W[None, :]) @ psi.T
        if np.any(bnd):
            bout += float(np.sum(Fout[bnd] * 0.5 * (g[bnd] @ GAUSS3_W)))
    c_new = c + dt * R / (poro[:, None] * grid.vol * MASS[None, :])
    return c_new, bout


def shock_detector(grid: Grid, c: np.ndarray, F: np.ndarray, s_D: np.ndarray) -> np.ndarray:
    """eta(e) of Section 3.4 (module docstring)."""
    fl, fr, fb, ft = _cell_faces(grid)
    h = np.hypot(grid.hx, grid.hy)
    eta = np.zeros(grid.n_cells)
    for side, Fs in enumerate((F[fl], F[fr], F[fb], F[ft])):
        r, t, sgn = _SIDES[side]
        Fout = sgn * Fs
        ln = grid.hy if r is not None else grid.hx
        own = _trace(c, side, np.zeros(1))[:, 0]  # trace at the face midpoint (traces are linear)
        nb = _neighbour(grid, side)
        other = np.empty(grid.n_cells)
        inside = nb >= 0
        other[inside] = _trace(c[nb[inside]], side ^ 1, np.zeros(1))[:, 0]
        other[~inside] = s_D[_boundary_index(grid, side)[~inside]]
        upstream = Fout < 0.0
        eta += np.where(upstream, np.abs(ln * (own - other)), 0.0)
    return eta / (0.08 * 2.0 * np.sqrt(h) * grid.vol)


def gradient_scale(g: float, d: float) -> float:
    """m_i of Section 3.4 from g_i and d_i (the three cases as printed)."""
    if g * d < 0.0 and abs(g) > 1e-8 and abs(d) > 1e-8:
        return 0.0
    if g * d > 0.0 and abs(g) > abs(d) and abs(g) > 1e-8 and abs(d) > 1e-8:
        return d / g
    return 1.0


def limit(grid: Grid, c: np.ndarray, F: np.ndarray, s_D: np.ndarray):
    """The limiter of Section 3.4. Returns (limited c, flagged mask); every
    cell is limited from the unlimited state of its neighbours."""
    eta = shock_detector(grid, c, F, s_D)
    vert = np.stack([c[:, 0] + a * c[:, 1] + b * c[:, 2] for a in (-1, 1) for b in (-1, 1)], axis=1)
    flagged = (eta > 1.0) | np.any((vert < 0.0) | (vert > 1.0), axis=1)
    out = c.copy()
    # g_i = grad s . (b_i - b_e): left -2 c1, right +2 c1, bottom -2 c2, top +2 c2
    for e in np.nonzero(flagged)[0]:
        ms = []
        for side in range(4):
            nb = _neighbour(grid, side)[e]
            if nb < 0:
                continue
            g = (-2.0 if side in (0, 2) else 2.0) * c[e, 1 if side < 2 else 2]
            ms.append(gradient_scale(g, c[nb, 0] - c[e, 0]))
        alpha = min(ms) if ms else 1.0
        out[e, 1:] = alpha * c[e, 1:]
    return out, flagged


def fine_step_dg(model, c: np.ndarray) -> dict:
    """Algorithm 1 with k = 1 for the saturation: pressure, fluxes (mobility at
    the cell means), DG step, limiter."""
    lam = model.mobility(c[:, 0])
    p = model.solve_pressure(lam)
    F = model.fluxes(p, lam)
    if model.dt_fixed is not None:
        dt = float(model.dt_fixed)
    else:
        dt = dg_time_step(model.grid, F, model.poro, model.Lf, model.cfl, model.dt_max)
    c_new, bout = dg_step(model.grid, c, F, model.poro, dt, model.s_D, model.eta_w, model.eta_o, model.law)
    c_lim, flagged = limit(model.grid, c_new, F, model.s_D)
    return dict(p=p, F=F, dt=dt, c_unlimited=c_new, c=c_lim, flagged=flagged, boundary_outflow=bout)
