"""Pins for mobilities, the upwind saturation step, the fine IMPES scheme and
the time-of-flight (Eqs. brooksCorey, frationalFlow, Definition 3,
Algorithm 1, Eq. timeOfFlight)."""
import json
import os

import numpy as np

from oracle.grid import Grid
from oracle.impes import FineModel
from oracle.physics import mobilities, frac_flow, max_frac_flow_slope
from oracle.tof import time_of_flight
from oracle.velocity import cell_outflows
from synth import make_problem

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")


def test_paper_profile_constant():
    """T9: the last wetting profile of the paper's benchmark is the constant
    lambda_w(1) = k_rw(1)/eta_w = 765.808 (linear k_rw), the first is 0."""
    c = json.load(open(GOLDEN))
    lw1, _, _ = mobilities(1.0, c["eta_w"], c["eta_o"], "linear")
    lw0, _, _ = mobilities(0.0, c["eta_w"], c["eta_o"], "linear")
    assert abs(float(lw1) - c["lambda_w_M"]) < 5e-4
    assert float(lw0) == c["lambda_w_1"]
    assert c["T_end"] / c["n_time_steps"] == 50.0
    assert c["grid"][0] * c["grid"][1] == c["n_cells"]


def test_frac_flow_properties_and_linear_slope():
    for law in ("linear", "corey"):
        s = np.linspace(0, 1, 1001)
        f = frac_flow(s, 1.0, 7.0, law)
        assert f[0] == 0.0 and f[-1] == 1.0 and np.all(np.diff(f) >= 0)
    # linear law: f' = a b / (a s + b (1 - s))^2 with a = 1/eta_w, b = 1/eta_o,
    # maximal at an end point: max(a/b, b/a)
    for ew, eo in ((1.0, 7.0), (3.0, 0.5), (0.00130581, 0.008)):
        exact = max(eo / ew, ew / eo)
        assert abs(max_frac_flow_slope(ew, eo, "linear") - exact) < 1e-6 * exact


def test_corey_slope_bruteforce():
    s = np.linspace(0, 1, 2_000_001)
    f = frac_flow(s, 1.0, 10.0, "corey")
    brute = np.max(np.diff(f) / np.diff(s))
    assert abs(max_frac_flow_slope(1.0, 10.0, "corey") - brute) < 1e-5 * brute


def _fine_run(prob, n_steps):
    m = FineModel.from_problem(prob)
    s = prob.s0.copy()
    hist = []
    for _ in range(n_steps):
        r = m.step(s)
        hist.append(r)
        s = r["s"]
    return m, s, hist


def test_mass_balance_and_bounds_fine():
    """T3 and T4: the water volume changes exactly by the boundary fluxes
    (interior face terms telescope), and 0 <= s <= 1 under CFL 0.5."""
    prob = make_problem("small")
    m, s, hist = _fine_run(prob, 30)
    vol = m.poro * m.grid.vol
    lhs = np.sum(vol * s) - np.sum(vol * prob.s0)
    rhs = -sum(h["dt"] * h["boundary_outflow"] for h in hist)
    assert abs(lhs - rhs) <= 1e-13 * abs(rhs)
    assert s.min() >= -1e-14 and s.max() <= 1.0 + 1e-14
    for h in hist:
        assert h["s"].min() >= -1e-14 and h["s"].max() <= 1.0 + 1e-14


def test_time_of_flight_uniform_flow():
    """Uniform flow in x: the upwind P0 time-of-flight of cell column i is
    exactly (i + 1) phi |e| / F."""
    nx, ny = 12, 5
    prob = make_problem("small").with_(nx=nx, ny=ny)
    g = Grid(nx, ny, 1.0, 1.0)
    F = np.zeros(g.n_faces)
    F[:g.nxf] = 0.37
    poro = np.full(g.n_cells, 0.2)
    tau = time_of_flight(g, F, poro)
    assert np.allclose(tau, (g.ci + 1) * 0.2 * g.vol / 0.37, rtol=1e-13)


def test_time_of_flight_residual_heterogeneous():
    """tau solves sum_f tau_up F_out = phi |e| on a heterogeneous fine
    velocity (checked cell by cell with the upwind rule)."""
    prob = make_problem("small")
    m = FineModel.from_problem(prob)
    lam = m.mobility(prob.s0)
    F = m.fluxes(m.solve_pressure(lam), lam)
    g = m.grid
    tau = time_of_flight(g, F, m.poro)
    res = np.zeros(g.n_cells)
    for f in g.interior:
        a, b = g.fe1[f], g.fe2[f]
        up = tau[a] if F[f] >= 0 else tau[b]
        res[a] += F[f] * up
        res[b] -= F[f] * up
    for k, f in enumerate(g.bface):
        Fo = F[f] * g.bsign[k]
        if Fo >= 0:
            res[g.bcell[k]] += Fo * tau[g.bcell[k]]
    assert np.allclose(res, m.poro * g.vol, rtol=1e-9)
    assert np.all(tau > 0)
