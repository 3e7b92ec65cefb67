"""Pins for the oracle's LRBMS offline phase and online step (Eqs.
parameterizedMob, leastSquaresFit, reducedSystem, Algorithm 2, Algorithm 3)."""
import numpy as np
import pytest

from oracle.grid import Coarse
from oracle.impes import FineModel
from oracle.offline import (build_offline, profiles_from_tof, gram_pinv, fit_theta,
                            orthonormalize, local_mass_rows, unit_function, restrict)
from oracle.physics import total_mobility
from oracle.reduced import online_step, online_run
from oracle.velocity import cell_outflows
from synth import make_problem, simplex_params, random_orthogonal


@pytest.fixture(scope="module")
def small_case():
    prob = make_problem("small")
    m = FineModel.from_problem(prob)
    co = Coarse(m.grid, prob.Sx, prob.Sy)
    off = build_offline(m, co, prob.s0, prob.n_steps, prob.M, kind="greedy",
                        train=simplex_params(48, prob.M, 11), cap=10, tol=1e-6)
    return prob, m, co, off


def test_profiles_definition_and_index():
    rng = np.random.default_rng(1)
    tau = rng.uniform(0, 2.0, 500)
    M, T = 8, 1.5
    P, idx = profiles_from_tof(tau, T, M, 0.1, 1.0)
    for e in range(len(tau)):
        for q in range(1, M + 1):
            if q == 1:
                want = 0.1
            elif q == M:
                want = 1.0
            else:
                want = 0.1 if tau[e] > (q - 1) * T / (M - 2) else 1.0
            assert P[q - 1, e] == want
            assert (P[q - 1, e] == 1.0) == (q >= idx[e])


def test_fit_matches_lstsq_bruteforce():
    """T8: theta = G^+ P lambda(s) gives the least-squares fitted mobility of
    numpy's lstsq (also for the rank-deficient profile sets of Algorithm 2)."""
    rng = np.random.default_rng(2)
    for trial in range(5):
        n, M = 40, 6
        tau = rng.uniform(0, 1, n)
        P, _ = profiles_from_tof(tau, 0.8, M, 0.2, 1.0)
        if trial % 2:
            P = rng.uniform(0.1, 1.0, (M, n))
        s = rng.uniform(0, 1, n)
        th = fit_theta(s, P, gram_pinv(P), 1.0, 5.0, "corey")
        lam = total_mobility(s, 1.0, 5.0, "corey")
        ref, *_ = np.linalg.lstsq(P.T, lam, rcond=None)
        assert np.allclose(th @ P, ref @ P, rtol=1e-11, atol=1e-13)
        if trial % 2:  # full rank: the coefficients themselves are unique
            assert np.allclose(th, ref, rtol=1e-8)


def test_fit_exact_for_uniform_saturation(small_case):
    prob, m, co, off = small_case
    for sval in (0.0, 0.3, 1.0):
        s = np.full(m.grid.n_cells, sval)
        th = fit_theta(s, off.P, off.Gp, m.eta_w, m.eta_o, m.law)
        assert np.allclose(th @ off.P, m.mobility(s), rtol=1e-12)


def test_gram_schmidt_local_orthonormality(small_case):
    prob, m, co, off = small_case
    mrow = local_mass_rows(m.grid, co.cx * co.cy)
    for E in range(co.n_sub):
        Ph = off.Phi[E]
        G = Ph.T @ (mrow[:, None] * Ph)
        assert np.abs(G - np.eye(Ph.shape[1])).max() < 1e-13
        assert np.allclose(Ph[:, 0], unit_function(m.grid, co.cx * co.cy))
    # rejection of a dependent extension
    v = Ph[:, 1] * 2.0 + Ph[:, 0]
    assert orthonormalize(v, [Ph[:, k] for k in range(Ph.shape[1])], mrow) is None


def test_greedy_error_decreases(small_case):
    hist = small_case[3].extra["greedy"]
    assert hist[-1] < 0.05 * hist[0]


def test_reduced_mass_balance(small_case):
    """T3 on the reduced path: interior face terms telescope for any
    velocity, so the balance is exact even though the reduced velocity is not
    locally conservative."""
    prob, m, co, off = small_case
    s, hist = online_run(m, off, prob.s0, 20)
    vol = m.poro * m.grid.vol
    lhs = np.sum(vol * s) - np.sum(vol * prob.s0)
    rhs = -sum(h["dt"] * h["boundary_outflow"] for h in hist)
    assert abs(lhs - rhs) <= 1e-13 * abs(rhs)


def test_snapshot_reproduction(small_case):
    """T5: with the fine solution for the current (exactly fitted) mobility in
    the local bases, the reduced pressure equals it (Galerkin, W_N in V_h)."""
    prob, m, co, _ = small_case
    s = np.full(m.grid.n_cells, 0.35)
    lam = m.mobility(s)
    p_fine = m.solve_pressure(lam)
    mrow = local_mass_rows(m.grid, co.cx * co.cy)
    Phi = []
    for E in range(co.n_sub):
        b = [unit_function(m.grid, co.cx * co.cy)]
        w = orthonormalize(restrict(co, p_fine, E), b, mrow)
        if w is not None:
            b.append(w)
        Phi.append(np.stack(b, axis=1))
    off = build_offline(m, co, prob.s0, prob.n_steps, prob.M, Phi=Phi)
    r = online_step(m, off, s)
    assert np.linalg.norm(r["p"] - p_fine) <= 1e-10 * np.linalg.norm(p_fine)
    # exact fit + unit functions: the reduced velocity is conservative per subdomain
    out = cell_outflows(m.grid, r["F"])
    per_sub = np.bincount(co.sub_of_cell, weights=out, minlength=co.n_sub)
    assert np.abs(per_sub).max() <= 1e-9 * np.abs(r["F"]).max()


def test_full_basis_equivalence():
    """T6: local bases spanning each subdomain's whole DG space and profiles
    that contain lambda(s^n) make one reduced step equal one fine step
    (p, F, s, dt)."""
    prob = make_problem("small").with_(nx=8, ny=8, Sx=2, Sy=2)
    from synth.fields import lognormal_field
    from synth.problems import default_bcs
    bc, pD, vN, sD = default_bcs(8, 8)
    prob = prob.with_(perm=lognormal_field(8, 8, 1.0, 1.0, 1.0, (0.2, 0.2), 4), poro=np.full(64, 0.2),
                      s0=np.zeros(64), bc_type=bc, p_D=pD, v_N=vN, s_D=sD)
    m = FineModel.from_problem(prob)
    co = Coarse(m.grid, 2, 2)
    rng = np.random.default_rng(8)
    s = rng.uniform(0, 1, 64)
    lam = m.mobility(s)
    P = np.stack([np.full(64, m.mobility(0.0)), lam, rng.uniform(0.1, 1.0, 64), np.full(64, m.mobility(1.0))])
    nE = 16
    Phi = [np.eye(3 * nE) for _ in range(4)]
    off = build_offline(m, co, prob.s0, 10, 4, Phi=Phi, P=P)
    r = online_step(m, off, s)
    f = m.step(s)
    for k in ("p", "F", "s"):
        assert np.linalg.norm(r[k] - f[k]) <= 1e-10 * np.linalg.norm(f[k]), k
    assert abs(r["dt"] - f["dt"]) <= 1e-10 * f["dt"]


def test_rotation_invariance(small_case):
    """T7: rotating every local basis by an orthogonal Q_E leaves p, F and s
    of the online step unchanged."""
    prob, m, co, off = small_case
    rng = np.random.default_rng(21)
    PhiR = [B @ random_orthogonal(B.shape[1], rng) for B in off.Phi]
    offR = build_offline(m, co, prob.s0, prob.n_steps, prob.M, Phi=PhiR)
    s = np.clip(np.random.default_rng(5).normal(0.3, 0.2, m.grid.n_cells), 0, 1)
    a = online_step(m, off, s)
    b = online_step(m, offR, s)
    for k in ("p", "F", "s"):
        assert np.linalg.norm(a[k] - b[k]) <= 1e-10 * np.linalg.norm(a[k]), k


def test_reduced_close_to_fine_early(small_case):
    """The reduced pressure of the first step (s = s0 = 0, exactly fitted)
    reproduces the fine pressure closely (greedy with the true error)."""
    prob, m, co, off = small_case
    a = online_step(m, off, prob.s0)
    f = m.step(prob.s0)
    assert np.linalg.norm(a["p"] - f["p"]) <= 1e-2 * np.linalg.norm(f["p"])


def test_fitted_velocity_variant():
    """The fitted-mobility velocity (reading R7's variant) uses
    sum_q theta_q Lambda^q in Definition 2. For a uniform saturation the fit
    is exact (T8), so both variants give the same fluxes to round-off; after
    the front has formed they differ, and the variant still conserves the
    water volume exactly (its fluxes are single-valued per face)."""
    from lrbms_cases import case
    from oracle.reduced import online_step
    prob, m, co, off = case("small", kind="snapshots")
    s_u = np.full(prob.n_cells, 0.4)
    a = online_step(m, off, s_u)
    b = online_step(m, off, s_u, velocity="fitted")
    assert np.linalg.norm(a["F"] - b["F"]) <= 1e-11 * np.linalg.norm(a["F"])
    s = prob.s0.copy()
    for _ in range(10):
        s = online_step(m, off, s)["s"]
    a = online_step(m, off, s)
    b = online_step(m, off, s, velocity="fitted")
    assert np.linalg.norm(a["F"] - b["F"]) > 1e-6 * np.linalg.norm(a["F"])
    vol = prob.poro * m.grid.vol
    dm = np.sum(vol * b["s"]) - np.sum(vol * s)
    assert abs(dm + b["dt"] * b["boundary_outflow"]) <= 1e-13 * abs(b["dt"] * b["boundary_outflow"])
