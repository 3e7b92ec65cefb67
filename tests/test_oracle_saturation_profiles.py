"""Pins for the profile variant of Section 6 (profiles from high-dimensional
saturation snapshots, Lambda^q = lambda(s_h^{n_q})): the profiles are the
mobilities of states of the fine trajectory, the least-squares fit of
Eq. leastSquaresFit is exact at those states, and with local bases that span
every subdomain's whole DG space a reduced step from such a state equals the
fine step (with threshold profiles it does not)."""
import numpy as np

from oracle.grid import Coarse
from oracle.impes import FineModel
from oracle.offline import build_offline, fit_theta, gram_pinv, saturation_profiles
from oracle.reduced import online_step
from synth import make_problem

N_STEPS, M = 6, 4


def _setup():
    from synth.fields import lognormal_field
    from synth.problems import default_bcs
    prob = make_problem("small").with_(nx=8, ny=8, Sx=2, Sy=2)
    bc, pD, vN, sD = default_bcs(8, 8)
    prob = prob.with_(perm=lognormal_field(8, 8, 1.0, 1.0, 1.0, (0.2, 0.2), 4), poro=np.full(64, 0.2),
                      s0=np.zeros(64), bc_type=bc, p_D=pD, v_N=vN, s_D=sD)
    m = FineModel.from_problem(prob)
    return prob, m


def test_profiles_are_mobilities_along_the_fine_trajectory():
    """Profile 1 is the uniform lambda(0) of s0 = 0 (1/eta_o for Corey), the
    last one lambda of the fine state after N_STEPS steps, and the ones in
    between lambda of the fine states at the rounded equal spacing."""
    prob, m = _setup()
    P = saturation_profiles(m, prob.s0, N_STEPS, M)
    assert P.shape == (M, 64)
    assert np.allclose(P[0], 1.0 / m.eta_o, rtol=1e-15, atol=0)
    states = [prob.s0]
    s = prob.s0
    for _ in range(N_STEPS):
        s = m.step(s)["s"]
        states.append(s)
    for q, n in enumerate((0, 2, 4, 6)):  # round(q * 6 / 3)
        assert np.array_equal(P[q], m.mobility(states[n])), q
    assert np.linalg.matrix_rank(P) == M


def test_fit_is_exact_at_the_snapshot_states():
    """theta = G^+ P lambda(s) reproduces lambda(s) when it is one of the
    profiles (linearly independent profiles: theta is the unit vector)."""
    prob, m = _setup()
    P = saturation_profiles(m, prob.s0, N_STEPS, M)
    Gp = gram_pinv(P)
    s = prob.s0
    for n in range(N_STEPS + 1):
        if n in (2, 4, 6):
            q = n // 2
            th = fit_theta(s, P, Gp, m.eta_w, m.eta_o, m.law)
            assert np.abs(th - np.eye(M)[q]).max() < 1e-10
            assert np.abs(th @ P - m.mobility(s)).max() < 1e-11 * np.abs(P[q]).max()
        s = m.step(s)["s"]


def test_full_basis_reduced_step_equals_fine_step_at_snapshot_states():
    prob, m = _setup()
    co = Coarse(m.grid, 2, 2)
    Phi = [np.eye(48) for _ in range(4)]
    P = saturation_profiles(m, prob.s0, N_STEPS, M)
    off = build_offline(m, co, prob.s0, 10, M, Phi=Phi, P=P)
    s = prob.s0
    for n in range(N_STEPS + 1):
        if n in (2, 4, 6):
            r, f = online_step(m, off, s), m.step(s)
            for k in ("p", "F", "s"):
                assert np.linalg.norm(r[k] - f[k]) <= 1e-10 * np.linalg.norm(f[k]), (n, k)
        s = m.step(s)["s"]
    # with the time-of-flight threshold profiles the same full-basis step differs
    off_t = build_offline(m, co, prob.s0, 10, M, Phi=Phi)
    s4 = m.run(prob.s0, 4)[0]
    r, f = online_step(m, off_t, s4), m.step(s4)
    assert np.linalg.norm(r["p"] - f["p"]) > 1e-6 * np.linalg.norm(f["p"])
