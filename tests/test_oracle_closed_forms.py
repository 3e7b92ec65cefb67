"""Closed-form pins for the oracle parts that the other tests only reach
through the oracle's own functions: the quadratic Corey law (Eq. brooksCorey),
the fractional flow (Eq. frationalFlow), the CFL time step (reading R12 of
the time-step rule) and the threshold profiles (Algorithm 2, step 1(c)).

Every expected value here is written out from the formula or computed by
hand; nothing is derived from ``oracle.physics`` or ``oracle.transport``, so
a wrong law (say k_rw = s), a wrong outflow sum (|F| instead of the positive
outflow) or an off-by-one threshold fails a test."""
import numpy as np
import pytest
from scipy.optimize import brentq

from oracle.grid import Grid
from oracle.impes import FineModel
from oracle.offline import profiles_from_tof
from oracle.physics import frac_flow, mobilities, relperm
from oracle.transport import cfl_dt
from synth import make_problem


# ---------------------------------------------------------------- Eq. brooksCorey
def test_corey_relperm_literal_values():
    """k_rw = s^2, k_ro = (1 - s)^2 at s = 0.3: 0.09 and 0.49 (by hand)."""
    krw, kro = relperm(0.3, "corey")
    assert abs(float(krw) - 0.09) < 1e-15
    assert abs(float(kro) - 0.49) < 1e-15
    krw, kro = relperm(0.3, "linear")
    assert abs(float(krw) - 0.3) < 1e-15 and abs(float(kro) - 0.7) < 1e-15


def test_corey_mobilities_literal_values():
    """eta_w = 1, eta_o = 10, s = 0.3: lambda_w = 0.09, lambda_o = 0.049,
    lambda = 0.139, f_w = 0.09 / 0.139 (hand arithmetic)."""
    lw, lo, lt = mobilities(0.3, 1.0, 10.0, "corey")
    assert abs(float(lw) - 0.09) < 1e-15
    assert abs(float(lo) - 0.049) < 1e-15
    assert abs(float(lt) - 0.139) < 1e-15
    assert abs(float(frac_flow(0.3, 1.0, 10.0, "corey")) - 0.09 / 0.139) < 1e-15
    # s = 0.5 with eta_o = 4: f_w = 0.25 / (0.25 + 0.0625) = 0.8
    assert abs(float(frac_flow(0.5, 1.0, 4.0, "corey")) - 0.8) < 1e-15


# ---------------------------------------------------------------- Buckley-Leverett, closed form
def _corey_fw(s, r):
    """Corey fractional flow with viscosity ratio r = eta_w / eta_o, written
    out: f = s^2 / (s^2 + r (1 - s)^2)."""
    return s * s / (s * s + r * (1.0 - s) ** 2)


def _corey_dfw(s, r):
    """Its derivative, by hand: f' = 2 r s (1 - s) / (s^2 + r (1 - s)^2)^2."""
    d = s * s + r * (1.0 - s) ** 2
    return 2.0 * r * s * (1.0 - s) / (d * d)


def test_welge_saturation_closed_form():
    """The Welge tangent f'(s*) s* = f(s*) of the Corey law has the closed
    form s* = sqrt(r / (1 + r)) (from s^2 + r (1-s)^2 = 2 r (1-s))."""
    for r in (0.5, 0.1, 2.0):
        ss = np.sqrt(r / (1.0 + r))
        assert abs(_corey_dfw(ss, r) * ss - _corey_fw(ss, r)) < 1e-14


def _bl_exact(x, Q, phi, r):
    """Buckley-Leverett profile for the injected volume Q per unit area into
    s = 0: rarefaction x = (Q / phi) f'(s) for s > s*, shock at
    x = Q f(s*) / (phi s*), from the closed forms above."""
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
def test_buckley_leverett_closed_form_convergence():
    """T2 against an exact profile that uses no oracle function: the fine
    scheme on the 1D strip (Corey law, viscosity ratio 2) converges in L1 to
    the closed-form Buckley-Leverett solution at equal injected volume."""
    errs = []
    for n in (100, 200, 400):
        prob = make_problem("strip", n=n, S=1)
        m = FineModel.from_problem(prob)
        r_visc = prob.eta_w / prob.eta_o
        s = prob.s0.copy()
        Q = 0.0
        while True:
            st = m.step(s)
            Q_next = Q + st["dt"] * st["F"][0] / m.grid.hy
            if Q_next > 0.12:
                break
            Q = Q_next
            s = st["s"]
        exact = _bl_exact(m.grid.xc, Q, 0.2, r_visc)
        errs.append(np.sum(np.abs(s - exact)) * m.grid.hx)
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert errs[-1] < 0.02, errs
    assert np.all(rates > 0.5), (errs, rates)


# ---------------------------------------------------------------- CFL step (reading R12)
def _uniform_faces(g: Grid, Fx: float, Fy: float) -> np.ndarray:
    F = np.zeros(g.n_faces)
    F[: g.nxf] = Fx
    F[g.nxf:] = Fy
    return F


def test_cfl_uniform_flow_in_x():
    """Uniform flow F in +x: every cell has one outflow face (right) of flux
    F, so dt = cfl phi |e| / (L_f F) exactly. Summing |F| over faces would
    count the inflow face too and halve dt."""
    g = Grid(6, 4, 1.0, 1.0)
    F = _uniform_faces(g, 0.37, 0.0)
    poro = np.full(g.n_cells, 0.2)
    Lf, cfl = 2.5, 0.5
    assert abs(cfl_dt(g, F, poro, Lf, cfl) - cfl * 0.2 * g.vol / (Lf * 0.37)) < 1e-15


def test_cfl_two_outflow_faces_and_porosity():
    """Flow up and to the right: each cell leaves through its right (0.37)
    and top (0.11) faces, outflow 0.48. With one cell of porosity 0.05 the
    minimum sits there: dt = cfl 0.05 |e| / (L_f 0.48). Flows entering
    through the left and bottom faces do not count."""
    g = Grid(5, 3, 2.0, 1.5)
    F = _uniform_faces(g, 0.37, 0.11)
    poro = np.full(g.n_cells, 0.2)
    poro[7] = 0.05
    Lf, cfl = 3.0, 0.25
    want = cfl * 0.05 * g.vol / (Lf * 0.48)
    assert abs(cfl_dt(g, F, poro, Lf, cfl) - want) < 1e-15 * want
    # reversing the flow keeps the outflow per cell (left and bottom faces)
    assert abs(cfl_dt(g, -F, poro, Lf, cfl) - want) < 1e-15 * want


def test_cfl_cap_and_no_flow():
    g = Grid(3, 3, 1.0, 1.0)
    poro = np.full(g.n_cells, 0.2)
    assert cfl_dt(g, np.zeros(g.n_faces), poro, 1.0, 0.5, dt_max=7.0) == 7.0
    F = _uniform_faces(g, 1.0, 0.0)
    assert cfl_dt(g, F, poro, 1.0, 0.5, dt_max=1e-6) == 1e-6


# ---------------------------------------------------------------- profiles (Algorithm 2, step 1(c))
def test_threshold_profiles_hand_example():
    """tau = (0.5, 1.5, 2.5, 3.5, 10), T = 6, M = 5: the thresholds of
    profiles q = 2, 3, 4 are (q - 1) T / (M - 2) = 2, 4, 6. A cell takes
    lambda(1) from the first q whose threshold it does not exceed, so the
    first lambda(1) index is 2, 2, 3, 3, 5 (worked by hand)."""
    tau = np.array([0.5, 1.5, 2.5, 3.5, 10.0])
    P, k = profiles_from_tof(tau, 6.0, 5, 0.1, 1.0)
    assert list(k) == [2, 2, 3, 3, 5]
    want = np.array([
        [0.1, 0.1, 0.1, 0.1, 0.1],   # q = 1: lambda(0)
        [1.0, 1.0, 0.1, 0.1, 0.1],   # q = 2: threshold 2
        [1.0, 1.0, 1.0, 1.0, 0.1],   # q = 3: threshold 4
        [1.0, 1.0, 1.0, 1.0, 0.1],   # q = 4: threshold 6
        [1.0, 1.0, 1.0, 1.0, 1.0],   # q = M: lambda(1)
    ])
    assert np.array_equal(P, want)
