"""Pins for the piecewise-linear DG saturation step and its limiter
(Definition 3 with k = 1; Section 3.4, Eq. limiterMain), against closed forms
and hand-worked values, not against the oracle's own functions."""
import numpy as np
import pytest
from scipy.optimize import brentq

from oracle.grid import Grid
from oracle.impes import FineModel
from oracle.transport_dg import dg_step, fine_step_dg, gradient_scale, limit, shock_detector
from synth import make_problem


def _uniform_x_flow(g: Grid, Fx: float) -> np.ndarray:
    F = np.zeros(g.n_faces)
    F[: g.nxf] = Fx
    return F


def test_uniform_state_in_uniform_flow_is_kept():
    """A uniform saturation in a divergence-free uniform flow (inflow carrying
    the same saturation) is a steady state of the scheme: every volume and
    face term cancels, to round-off."""
    g = Grid(8, 5, 1.0, 1.0)
    c = np.zeros((g.n_cells, 3))
    c[:, 0] = 0.37
    s_D = np.full(2 * g.nx + 2 * g.ny, 0.37)
    cn, _ = dg_step(g, c, _uniform_x_flow(g, 0.3 * g.hy), np.full(g.n_cells, 0.2), 1e-3, s_D, 1.0, 5.0, "corey")
    assert np.abs(cn - c).max() < 1e-15


def test_linear_profile_is_advected_exactly():
    """f(s) = s (linear law, equal viscosities): a linear profile s = a + b x in
    a uniform flow u moves exactly, s(x, dt) = a + b (x - u dt): the cell
    means drop by b u dt / phi, the slopes stay (one explicit Euler step is
    exact because the time derivative is constant)."""
    g = Grid(10, 4, 1.0, 1.0)
    a, b, u, phi, dt = 0.2, 0.5, 0.7, 0.25, 0.01
    c = np.zeros((g.n_cells, 3))
    c[:, 0] = a + b * g.xc
    c[:, 1] = b * g.hx / 2.0
    s_D = np.zeros(2 * g.nx + 2 * g.ny)
    s_D[: g.ny] = a  # inflow at x = 0 carries s(0)
    cn, _ = dg_step(g, c, _uniform_x_flow(g, u * g.hy), np.full(g.n_cells, phi), dt, s_D, 1.0, 1.0, "linear")
    assert np.abs(cn[:, 0] - (c[:, 0] - b * u * dt / phi)).max() < 1e-14
    assert np.abs(cn[:, 1:] - c[:, 1:]).max() < 1e-14
    lim, flagged = limit(g, cn, _uniform_x_flow(g, u * g.hy), s_D)
    # only the inflow column is flagged (the fixed s_D now differs from the
    # moved profile's trace); a linear profile has m_i = 1 everywhere, so the
    # limiter changes nothing
    assert not flagged[g.ci > 0].any()
    assert np.abs(lim - cn).max() < 1e-14


def test_gradient_scales_as_printed():
    """The three cases of m_i (Section 3.4), worked by hand."""
    assert gradient_scale(0.4, -0.1) == 0.0           # opposite signs: flatten
    assert gradient_scale(0.4, 0.1) == 0.25           # overshoot: d/g
    assert gradient_scale(0.1, 0.4) == 1.0            # |g| <= |d|: keep
    assert gradient_scale(1e-9, -0.3) == 1.0          # tiny g: keep
    assert gradient_scale(0.3, 1e-9) == 1.0           # tiny d: keep


def test_limiter_flattens_a_local_extremum_and_keeps_means():
    """Worked by hand: three unit cells in a row, means 0.1, 0.5, 0.3, the
    centre with slope c1 = 0.6 (vertex values -0.1 and 1.1, outside [0, 1],
    so it is flagged; its upstream jump 0.2 - ... gives eta = 0.2 /
    (0.16 2^(1/4)) = 1.0511 > 1 as well). m_left: g = -2 c1 = -1.2 and
    d = -0.4 share a sign with |g| > |d| -> 1/3; m_right: g = 1.2 and
    d = -0.2 have opposite signs -> 0. The slope is removed; every mean is
    kept."""
    g = Grid(3, 1, 3.0, 1.0)
    c = np.array([[0.1, 0.0, 0.0], [0.5, 0.6, 0.0], [0.3, 0.0, 0.0]])
    F = np.zeros(g.n_faces)
    F[: g.nxf] = 1.0  # flow in +x: the left faces are upstream
    s_D = np.full(2 * g.nx + 2 * g.ny, 0.1)
    eta = shock_detector(g, c, F, s_D)
    assert abs(eta[1] - 0.2 / (0.16 * 2.0 ** 0.25)) < 1e-14
    lim, flagged = limit(g, c, F, s_D)
    # the right cell is flagged too (its upstream jump 0.3 - 1.1), but has no
    # slope to limit
    assert list(flagged) == [False, True, True]
    assert lim[1, 1] == 0.0 and lim[1, 0] == 0.5
    assert np.array_equal(lim[:, 0], c[:, 0]) and np.array_equal(lim[2], c[2])


def test_limiter_scales_an_overshooting_slope():
    """Means 0.0, 0.5, 1.0 rising in x with the centre's slope c1 = 0.6
    (vertex values -0.1 and 1.1: flagged): g_left = -1.2, d_left = -0.5
    -> 0.5/1.2; g_right = 1.2, d_right = 0.5 -> 0.5/1.2; the slope becomes
    0.6 * 5/12 = 0.25 (vertex values 0.25 and 0.75)."""
    g = Grid(3, 1, 3.0, 1.0)
    c = np.array([[0.0, 0.0, 0.0], [0.5, 0.6, 0.0], [1.0, 0.0, 0.0]])
    F = np.zeros(g.n_faces)
    F[: g.nxf] = 1.0
    s_D = np.zeros(2 * g.nx + 2 * g.ny)
    lim, flagged = limit(g, c, F, s_D)
    assert flagged[1]
    assert abs(lim[1, 1] - 0.25) < 1e-15 and lim[1, 0] == 0.5


def test_detector_value_by_hand():
    """eta for one upstream face: |int_f [s] ds| / (0.08 d sqrt(h) |e|) with
    d = 2, h = diam(e): unit square cells, jump 0.01 over a face of length
    1 -> 0.01 / (0.16 sqrt(sqrt 2))."""
    g = Grid(2, 1, 2.0, 1.0)
    c = np.array([[0.30, 0.0, 0.0], [0.31, 0.0, 0.0]])
    F = np.zeros(g.n_faces)
    F[: g.nxf] = 1.0
    s_D = np.full(2 * g.nx + 2 * g.ny, 0.30)
    eta = shock_detector(g, c, F, s_D)
    assert abs(eta[1] - 0.01 / (0.16 * np.sqrt(np.sqrt(2.0)))) < 1e-14
    assert eta[0] == 0.0  # its upstream face carries s_D = its own value


def test_dg_mass_balance_and_bounds_fine():
    """T3 for the DG scheme with the limiter: the water volume (cell means)
    changes by exactly the boundary fluxes; the limited means stay in
    [0, 1] up to round-off on the 32x32 benchmark."""
    prob = make_problem("small")
    m = FineModel.from_problem(prob)
    c = np.zeros((prob.n_cells, 3))
    vol = m.poro * m.grid.vol
    out = 0.0
    for _ in range(15):
        r = fine_step_dg(m, c)
        out += r["dt"] * r["boundary_outflow"]
        assert np.array_equal(r["c"][:, 0], r["c_unlimited"][:, 0])  # the limiter keeps the means
        c = r["c"]
    assert abs((np.sum(vol * c[:, 0]) - 0.0) + out) <= 1e-13 * abs(out)
    assert c[:, 0].min() > -1e-3 and c[:, 0].max() < 1.0 + 1e-3


def _corey_fw(s, r):
    return s * s / (s * s + r * (1.0 - s) ** 2)


def _corey_dfw(s, r):
    d = s * s + r * (1.0 - s) ** 2
    return 2.0 * r * s * (1.0 - s) / (d * d)


def _bl_exact(x, Q, phi, r):
    ss = np.sqrt(r / (1.0 + r))
    xs = Q * _corey_fw(ss, r) / (phi * ss)
    out = np.zeros_like(x)
    for k, xx in enumerate(x):
        if xx >= xs:
            continue
        target = xx * phi / Q
        out[k] = 1.0 if target <= _corey_dfw(1.0 - 1e-12, r) else brentq(
            lambda s: _corey_dfw(s, r) - target, ss, 1.0 - 1e-12, xtol=1e-14)
    return out


@pytest.mark.slow
def test_dg_buckley_leverett_convergence():
    """T2 for the DG scheme with the limiter: the cell means converge in L1 to
    the closed-form Buckley-Leverett profile (Welge shock) on the 1D strip."""
    errs = []
    for n in (50, 100, 200):
        prob = make_problem("strip", n=n, S=1)
        m = FineModel.from_problem(prob)
        r_visc = prob.eta_w / prob.eta_o
        c = np.zeros((n, 3))
        Q = 0.0
        while True:
            st = fine_step_dg(m, c)
            Q_next = Q + st["dt"] * st["F"][0] / m.grid.hy
            if Q_next > 0.12:
                break
            Q = Q_next
            c = st["c"]
        exact = _bl_exact(m.grid.xc, Q, 0.2, r_visc)
        errs.append(np.sum(np.abs(c[:, 0] - exact)) * m.grid.hx)
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert errs[-1] < 0.02, errs
    assert np.all(rates > 0.5), (errs, rates)


def test_reduced_dg_step_mass_balance():
    """The reduced online step with the DG transport conserves the water
    volume exactly (the reduced fluxes are single-valued per face)."""
    from lrbms_cases import case
    from oracle.reduced import online_step_dg
    prob, m, co, off = case("small", kind="snapshots")
    c = np.zeros((prob.n_cells, 3))
    vol = m.poro * m.grid.vol
    out = 0.0
    for _ in range(6):
        r = online_step_dg(m, off, c)
        out += r["dt"] * r["boundary_outflow"]
        c = r["c"]
    assert abs(np.sum(vol * c[:, 0]) + out) <= 1e-13 * abs(out)


@pytest.mark.parametrize("axis", [0, 1])
def test_step_at_a_jump_matches_the_textbook_p1_scheme(axis):
    """Linear advection (f(s) = s) with uniform speed u along an axis: the
    upwind P1-DG equations on cell j with Legendre coefficients (mean c0,
    slope c1 along the flow) are, written out by hand,
        h dc0/dt = -u [(c0_j + c1_j) - (c0_{j-1} + c1_{j-1})],
        (h/3) dc1/dt = 2 u c0_j - u (c0_j + c1_j) - u (c0_{j-1} + c1_{j-1}),
    times 1/phi. For a unit step from s = 1 (upstream cell) to s = 0 the
    cell right of the jump gets c0 = u dt / (phi h) and c1 = -3 u dt /
    (phi h) after one explicit Euler step."""
    n = 6
    g = Grid(n, 1, 1.0, 1.0 / n) if axis == 0 else Grid(1, n, 1.0 / n, 1.0)
    u, phi, dt = 0.8, 0.3, 1e-3
    h = 1.0 / n
    c = np.zeros((g.n_cells, 3))
    c[: n // 2, 0] = 1.0  # upstream half full
    F = np.zeros(g.n_faces)
    if axis == 0:
        F[: g.nxf] = u * g.hy
    else:
        F[g.nxf:] = u * g.hx
    s_D = np.ones(2 * g.nx + 2 * g.ny)
    cn, _ = dg_step(g, c, F, np.full(g.n_cells, phi), dt, s_D, 1.0, 1.0, "linear")
    j = n // 2
    k = 1 + axis  # slope coefficient along the flow
    assert abs(cn[j, 0] - u * dt / (phi * h)) < 1e-14
    assert abs(cn[j, k] - (-3.0 * u * dt / (phi * h))) < 1e-13
    assert abs(cn[j, 3 - k]) < 1e-15
    # the upstream neighbour sees s = 1 on both sides: nothing changes there
    assert abs(cn[j - 1, 0] - 1.0) < 1e-14 and abs(cn[j - 1, k]) < 1e-13
