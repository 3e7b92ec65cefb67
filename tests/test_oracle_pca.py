"""Pins for the optional compression of Algorithm 2 (step 3, principal
component analysis of the restricted snapshots) and for the greedy's record
of the chosen snapshots, on constructed sets with known components."""
import numpy as np

from oracle.grid import Coarse, Grid
from oracle.offline import local_mass_rows, orthonormalize, pca_bases


def _orthonormal_functions(g, k, seed):
    m = local_mass_rows(g, g.n_cells)
    rng = np.random.default_rng(seed)
    q = []
    while len(q) < k:
        w = orthonormalize(rng.standard_normal(3 * g.n_cells), q, m)
        if w is not None:
            q.append(w)
    return np.stack(q, axis=1), m


def _snapshots(g, sig, n, seed):
    """n snapshots s_i = sum_k U_ik sig_k q_k with U (n x r) orthonormal
    columns: their L2 Gram matrix is U diag(sig^2) U^T, eigenvalues sig^2."""
    q, m = _orthonormal_functions(g, len(sig), seed)
    U, _ = np.linalg.qr(np.random.default_rng(seed + 1).standard_normal((n, len(sig))))
    S = (q * np.asarray(sig)[None, :]) @ U.T  # (3 n_cells, n)
    return [S[:, i] for i in range(n)], q, m


def test_pca_recovers_a_low_rank_set():
    """Three components with energies 1, 1e-2, 1e-4 behind 7 snapshots on one
    subdomain: a tiny tolerance keeps exactly the 3 components (each mode is
    +-q_k), the modes are L2-orthonormal and every snapshot is reproduced."""
    g = Grid(4, 3, 1.0, 1.0)
    co = Coarse(g, 1, 1)
    snaps, q, m = _snapshots(g, [1.0, 0.1, 0.01], 7, 5)
    # the coarse grid's local order equals the global order for one subdomain
    (Phi,) = pca_bases(co, snaps, g, 1e-12)
    assert Phi.shape[1] == 3
    G = Phi.T @ (m[:, None] * Phi)
    assert np.abs(G - np.eye(3)).max() < 1e-12
    overlap = np.abs(q.T @ (m[:, None] * Phi))
    assert np.abs(overlap - np.eye(3)).max() < 1e-9
    for s in snaps:
        proj = Phi @ (Phi.T @ (m * s))
        assert np.linalg.norm(proj - s) < 1e-10 * np.linalg.norm(s)


def test_pca_energy_criterion():
    """Discarded energy fraction at most eps^2: with energies 1, 1e-2, 1e-4
    (total 1.0101) eps^2 = 1.2e-4 / 1.0101 drops only the last component,
    eps = 0.5 drops both small ones, and the cap limits the count."""
    g = Grid(4, 3, 1.0, 1.0)
    co = Coarse(g, 1, 1)
    snaps, _, _ = _snapshots(g, [1.0, 0.1, 0.01], 7, 9)
    assert pca_bases(co, snaps, g, np.sqrt(1.2e-4 / 1.0101))[0].shape[1] == 2
    assert pca_bases(co, snaps, g, np.sqrt(0.9e-4 / 1.0101))[0].shape[1] == 3
    assert pca_bases(co, snaps, g, 0.5)[0].shape[1] == 1
    assert pca_bases(co, snaps, g, 1e-12, max_size=2)[0].shape[1] == 2


def test_greedy_records_the_chosen_snapshots():
    """The compression uses the snapshots the greedy selected (the set Psi of
    Algorithm 2, step 2(d)), one per extension step. Below the cap
    every greedy basis contains the restrictions of those snapshots, so the
    compressed modes lie in the span of the uncompressed basis and are
    L2-orthonormal; at a tiny tolerance they reproduce every snapshot."""
    from oracle.impes import FineModel
    from oracle.offline import build_offline, fine_solution, restrict
    from synth import make_problem, simplex_params
    prob = make_problem("rect", n=(24, 16), S=(3, 2))
    m = FineModel.from_problem(prob)
    co = Coarse(m.grid, prob.Sx, prob.Sy)
    train = simplex_params(12, prob.M, 11)
    kw = dict(kind="greedy", train=train, cap=8, tol=1e-3)
    plain = build_offline(m, co, prob.s0, prob.n_steps, prob.M, **kw)
    comp = build_offline(m, co, prob.s0, prob.n_steps, prob.M, pca_eps=1e-10, **kw)
    hist, chosen = comp.extra["greedy"], comp.extra["chosen"]
    assert len(chosen) >= 2 and len(chosen) in (len(hist), len(hist) - 1)
    assert np.all(plain.N_E < 8)  # below the cap: every snapshot extended every basis
    mass = local_mass_rows(m.grid, co.cx * co.cy)
    snaps = [fine_solution(m, plain.P, train[k]) for k in chosen]
    for E in range(co.n_sub):
        B, Q = comp.Phi[E], plain.Phi[E]
        assert 1 <= B.shape[1] <= len(chosen)
        G = B.T @ (mass[:, None] * B)
        assert np.abs(G - np.eye(B.shape[1])).max() < 1e-12
        inside = Q @ (Q.T @ (mass[:, None] * B))
        assert np.abs(inside - B).max() < 1e-8 * np.abs(B).max()
        for s in snaps:
            v = restrict(co, s, E)
            proj = B @ (B.T @ (mass * v))
            assert np.sqrt((proj - v) @ (mass * (proj - v))) <= 1e-8 * np.sqrt(v @ (mass * v))
