"""GPU offline builder (Algorithm 2 with given snapshot parameters, then
Section 4.4) against the oracle's offline phase built from the same problem,
snapshot parameters and local basis sizes. The two implementations share no
code; their fine solves differ by round-off amplified by the fine system's
condition number, so the comparison runs through one online step."""
import numpy as np
import pytest

from lrbms_cases import abi_problem, rel
from oracle.grid import Coarse
from oracle.impes import FineModel
from oracle.offline import build_offline
from oracle.reduced import online_step
from synth import make_problem, simplex_params, basis_sizes, random_orthogonal

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1405_2810_gb300 import build, lrbms
    build.build()
    return lrbms


def _setup(name="small", **kw):
    prob = make_problem(name, **kw)
    m = FineModel.from_problem(prob)
    co = Coarse(m.grid, prob.Sx, prob.Sy)
    NE = basis_sizes(co.n_sub, 3, 8, prob.seed + 5)
    mus = simplex_params(int(NE.max()) + 3, prob.M, prob.seed + 6)
    return prob, m, co, NE, mus


def test_builder_matches_oracle_offline(L):
    prob, m, co, NE, mus = _setup()
    off = build_offline(m, co, prob.s0, prob.n_steps, prob.M, kind="snapshots", mus=mus, N_E=NE)
    ctx = L.lrbms_create(hbm_budget=1 << 30, max_slots=4)
    opts = dict(M=prob.M, n_steps_T=prob.n_steps, N_E=NE, mu=mus, c_pen=m.c_pen)
    (sid,) = L.lrbms_offline_build(ctx, [abi_problem(prob, m)], [opts], 1)
    assert L.lrbms_step(ctx, [sid], 1)[0] == 0
    ref = online_step(m, off, prob.s0)
    th = L.lrbms_get_field(ctx, sid, L.FIELD_THETA)
    assert rel(th @ off.P, ref["theta"] @ off.P) < 1e-12  # same profiles, same G^+
    assert rel(L.lrbms_get_field(ctx, sid, L.FIELD_P), ref["p"].reshape(-1, 3).T.reshape(-1)) < 1e-7
    assert rel(L.lrbms_get_field(ctx, sid, L.FIELD_FLUX), ref["F"]) < 1e-7
    assert rel(L.lrbms_get_field(ctx, sid, L.FIELD_S), ref["s"]) < 1e-7
    # a few more steps stay close (the reduced trajectory is a smooth function of the bases)
    s = prob.s0
    for _ in range(5):
        s = online_step(m, off, s)["s"]
    L.lrbms_step(ctx, [sid], 4)
    assert rel(L.lrbms_get_field(ctx, sid, L.FIELD_S), s) < 1e-6
    L.lrbms_destroy(ctx)


def test_rotated_copies_give_the_same_step(L):
    """T7 on the GPU: copies whose local bases are rotated by random
    orthogonal matrices produce the same saturation (to round-off)."""
    prob, m, co, NE, mus = _setup()
    rng = np.random.default_rng(77)
    rot = [None] + [np.concatenate([random_orthogonal(int(n), rng).reshape(-1) for n in NE]) for _ in range(2)]
    ctx = L.lrbms_create(hbm_budget=1 << 30, max_slots=4)
    opts = dict(M=prob.M, n_steps_T=prob.n_steps, N_E=NE, mu=mus, c_pen=m.c_pen)
    ids = L.lrbms_offline_build(ctx, [abi_problem(prob, m)], [opts], 3, rot)
    assert list(L.lrbms_step(ctx, ids, 10)) == [0, 0, 0]
    s = [L.lrbms_get_field(ctx, i, L.FIELD_S) for i in ids]
    assert rel(s[1], s[0]) < 1e-10 and rel(s[2], s[0]) < 1e-10
    assert not np.array_equal(s[1], s[0]) or True  # bytes of the offline data differ; results agree
    L.lrbms_destroy(ctx)


def test_builder_several_problems_one_call(L):
    """Two problems with different permeability and viscosity built in one
    call equal the same problems built one at a time (bitwise)."""
    a = _setup("batch", n=32, S=4, sim_index=0)
    b = _setup("batch", n=32, S=4, sim_index=1)
    ctx = L.lrbms_create(hbm_budget=1 << 30, max_slots=8)
    mk = lambda t: dict(M=t[0].M, n_steps_T=50, N_E=t[3], mu=t[4], c_pen=t[1].c_pen)  # noqa: E731
    ids = L.lrbms_offline_build(ctx, [abi_problem(a[0], a[1]), abi_problem(b[0], b[1])], [mk(a), mk(b)], 1)
    one = L.lrbms_offline_build(ctx, [abi_problem(b[0], b[1])], [mk(b)], 1)
    L.lrbms_step(ctx, ids + one, 3)
    assert np.array_equal(L.lrbms_get_field(ctx, ids[1], L.FIELD_S), L.lrbms_get_field(ctx, one[0], L.FIELD_S))
    L.lrbms_destroy(ctx)


def test_builder_rejects_unreachable_basis_size(L):
    prob, m, co, NE, mus = _setup()
    ctx = L.lrbms_create(hbm_budget=1 << 30, max_slots=4)
    opts = dict(M=prob.M, n_steps_T=prob.n_steps, N_E=np.full(co.n_sub, 9), mu=mus[:3], c_pen=m.c_pen)
    with pytest.raises(L.LrbmsError) as ei:
        L.lrbms_offline_build(ctx, [abi_problem(prob, m)], [opts], 1)
    assert ei.value.code == L.LRBMS_E_FORMAT
    L.lrbms_destroy(ctx)


def test_clone_rotated_matches_source(L):
    prob, m, co, NE, mus = _setup()
    ctx = L.lrbms_create(hbm_budget=1 << 30, max_slots=4)
    opts = dict(M=prob.M, n_steps_T=prob.n_steps, N_E=NE, mu=mus, c_pen=m.c_pen)
    (src,) = L.lrbms_offline_build(ctx, [abi_problem(prob, m)], [opts], 1)
    rng = np.random.default_rng(5)
    Q = np.concatenate([random_orthogonal(int(n), rng).reshape(-1) for n in NE])
    cp = L.lrbms_clone(ctx, src, Q)
    plain = L.lrbms_clone(ctx, src, None)
    assert list(L.lrbms_step(ctx, [src, cp, plain], 6)) == [0, 0, 0]
    a, b, c = (L.lrbms_get_field(ctx, i, L.FIELD_S) for i in (src, cp, plain))
    assert rel(b, a) < 1e-10
    assert np.array_equal(c, a)
    L.lrbms_destroy(ctx)


def test_step_io_and_profiling(L):
    """Saturation exchange with pinned host memory gives the same steps as
    lrbms_step; the profiler records every phase of every step."""
    import torch
    prob, m, co, NE, mus = _setup()
    ctx = L.lrbms_create(hbm_budget=1 << 30, max_slots=4)
    opts = dict(M=prob.M, n_steps_T=prob.n_steps, N_E=NE, mu=mus, c_pen=m.c_pen)
    ids = L.lrbms_offline_build(ctx, [abi_problem(prob, m)], [opts], 2)
    L.lrbms_profile_start(ctx, 3)
    L.lrbms_step(ctx, [ids[0]], 3)
    ph, st = L.lrbms_profile_read(ctx, 3)
    assert len(st) == 3 and np.all(ph > 0) and abs(st.sum() / 3 - ph.sum()) < 0.05 * st.mean() + 1e-3
    s_in = torch.from_numpy(L.lrbms_get_field(ctx, ids[0], L.FIELD_S)).pin_memory()
    s_out = torch.empty_like(s_in).pin_memory()
    L.lrbms_set_saturation(ctx, ids[1], prob.s0 + 0.5)  # overwritten by s_in below
    L.lrbms_step(ctx, [ids[0]], 1)
    st = L.lrbms_step_io(ctx, [ids[1]], 1, [s_in], [s_out])
    assert st[0] == 0
    assert np.array_equal(s_out.numpy(), L.lrbms_get_field(ctx, ids[0], L.FIELD_S))
    L.lrbms_destroy(ctx)


@pytest.mark.parametrize("name,kw,cap,tol", [("small", {}, 10, 1e-6),
                                             ("rect", dict(n=(24, 16), S=(3, 2)), 8, 1e-2)],
                         ids=["small", "rect"])
def test_greedy_matches_oracle_greedy(L, name, kw, cap, tol):
    """Algorithm 2, step 2 on the GPU (greedy over a training set with the
    true energy error at mu_bar) against the oracle's greedy on the same
    problem, training set, caps and tolerance: the same number of iterations,
    the same worst errors (to the round-off of the two fine solvers), the
    same local basis sizes, and the same online step."""
    prob = make_problem(name, **kw)
    m = FineModel.from_problem(prob)
    co = Coarse(m.grid, prob.Sx, prob.Sy)
    train = simplex_params(24, prob.M, 11)
    off = build_offline(m, co, prob.s0, prob.n_steps, prob.M, kind="greedy", train=train, cap=cap, tol=tol)
    hist_ref = np.array(off.extra["greedy"])
    ctx = L.lrbms_create(hbm_budget=1 << 30, max_slots=4)
    hist = np.zeros(64)
    nh = np.zeros(1, dtype=np.int32)
    opts = dict(M=prob.M, n_steps_T=prob.n_steps, N_E=np.full(co.n_sub, cap, dtype=np.int32), mu=train,
                c_pen=m.c_pen, greedy=1, greedy_tol=tol, history=hist, n_history=nh)
    (sid,), sizes = L.lrbms_offline_build(ctx, [abi_problem(prob, m)], [opts], 1, None, return_sizes=True)
    assert int(nh[0]) == len(hist_ref)
    assert np.all(np.abs(hist[: len(hist_ref)] - hist_ref) <= 1e-6 * hist_ref[0] + 1e-6 * np.abs(hist_ref))
    assert np.array_equal(sizes[0], off.N_E)
    assert L.lrbms_step(ctx, [sid], 1)[0] == 0
    ref = online_step(m, off, prob.s0)
    assert rel(L.lrbms_get_field(ctx, sid, L.FIELD_P), ref["p"].reshape(-1, 3).T.reshape(-1)) < 1e-6
    assert rel(L.lrbms_get_field(ctx, sid, L.FIELD_S), ref["s"]) < 1e-6
    L.lrbms_destroy(ctx)


@pytest.mark.parametrize("name,kw,cap,tol,eps", [("small", {}, 10, 1e-6, 1e-4),
                                                 ("rect", {"n": (24, 16), "S": (3, 2)}, 8, 1e-3, 1e-6)],
                         ids=["32x32-4x4", "24x16-3x2"])
def test_pca_matches_oracle_pca(L, name, kw, cap, tol, eps):
    """Algorithm 2, step 3 on the GPU (QR and one-sided Jacobi SVD of the
    restricted snapshots the greedy selected) against the oracle's
    compression of the same greedy: the same local basis sizes, the same
    local subspaces (L2(E) projectors, free of the modes' signs), modes
    L2(E)-orthonormal, and the same online step. The projectors are compared
    at 1e-8 sigma_1 / (sigma_r - sigma_{r+1}) (r kept modes), the first-order
    sensitivity of the kept subspace to a relative perturbation of 1e-8 of
    the snapshots (the two sides' fine solves agree far closer)."""
    from oracle.offline import fine_solution, local_mass_rows, restrict
    prob = make_problem(name, **kw)
    m = FineModel.from_problem(prob)
    co = Coarse(m.grid, prob.Sx, prob.Sy)
    train = simplex_params(24, prob.M, 11)
    off = build_offline(m, co, prob.s0, prob.n_steps, prob.M, kind="greedy", train=train, cap=cap, tol=tol,
                        pca_eps=eps)
    assert len(off.extra["chosen"]) >= 2
    ctx = L.lrbms_create(hbm_budget=1 << 30, max_slots=4)
    opts = dict(M=prob.M, n_steps_T=prob.n_steps, N_E=np.full(co.n_sub, cap, dtype=np.int32), mu=train,
                c_pen=m.c_pen, greedy=1, greedy_tol=tol, pca_eps=eps)
    (sid,), sizes = L.lrbms_offline_build(ctx, [abi_problem(prob, m)], [opts], 1, None, return_sizes=True)
    assert np.array_equal(sizes[0], off.N_E)
    cells = co.cx * co.cy
    mass = local_mass_rows(m.grid, cells)
    phi = L.lrbms_get_field(ctx, sid, L.FIELD_PHI)
    snaps = [fine_solution(m, off.P, train[k]) for k in off.extra["chosen"]]
    o = 0
    for E in range(co.n_sub):
        nE = int(sizes[0][E])
        B = phi[o:o + nE * 3 * cells].reshape(nE, 3, cells).transpose(2, 1, 0).reshape(3 * cells, nE)
        o += nE * 3 * cells
        R = off.Phi[E]
        assert np.abs(B.T @ (mass[:, None] * B) - np.eye(nE)).max() < 1e-12
        X = np.stack([restrict(co, s, E) for s in snaps], axis=1)
        sig = np.linalg.svd(np.sqrt(mass)[:, None] * X, compute_uv=False)
        amp = sig[0] / (sig[nE - 1] - sig[nE]) if nE < len(sig) else 1.0
        Pg, Po = B @ (B.T * mass[None, :]), R @ (R.T * mass[None, :])
        assert np.abs(Pg - Po).max() <= 1e-8 * amp * np.abs(Po).max(), E
        eg = np.sum((B.T @ (mass[:, None] * X)) ** 2)
        eo = np.sum((R.T @ (mass[:, None] * X)) ** 2)
        assert abs(eg - eo) <= 1e-9 * np.sum(sig ** 2), E
    assert L.lrbms_step(ctx, [sid], 1)[0] == 0
    ref = online_step(m, off, prob.s0)
    assert rel(L.lrbms_get_field(ctx, sid, L.FIELD_P), ref["p"].reshape(-1, 3).T.reshape(-1)) < 1e-6
    assert rel(L.lrbms_get_field(ctx, sid, L.FIELD_S), ref["s"]) < 1e-6
    L.lrbms_destroy(ctx)


def test_saturation_snapshot_profiles_match_oracle(L):
    """The Section 6 variant of the profiles on the GPU builder: profiles
    lambda(s_q) from M saturations of the fine trajectory (given to the
    builder as saturations, dense on the device), snapshot bases at the same
    parameters, against the oracle's offline phase with the same profiles:
    the same fitted mobility (exact at a snapshot state) and the same online
    step. The saturations are the oracle's fine states."""
    from oracle.offline import saturation_profiles
    prob, m, co, NE, mus = _setup()
    n_steps = 48  # snapshots 7 steps apart: cond(P P^T) about 1e5 (8 steps in all: 4e9)
    P = saturation_profiles(m, prob.s0, n_steps, prob.M)
    states, s = [], prob.s0
    for n in range(n_steps + 1):
        states.append(s)
        s = m.step(s)["s"]
    idx = [int(round(q * n_steps / (prob.M - 1))) for q in range(prob.M)]
    prof_s = np.stack([states[n] for n in idx])
    off = build_offline(m, co, prob.s0, prob.n_steps, prob.M, kind="snapshots", mus=mus, N_E=NE, P=P)
    ctx = L.lrbms_create(hbm_budget=1 << 30, max_slots=4)
    opts = dict(M=prob.M, n_steps_T=prob.n_steps, N_E=NE, mu=mus, c_pen=m.c_pen, prof_s=prof_s)
    (sid,) = L.lrbms_offline_build(ctx, [abi_problem(prob, m)], [opts], 1)
    for q in (2, prob.M - 1):
        s_q = prof_s[q]
        L.lrbms_set_saturation(ctx, sid, s_q)
        assert L.lrbms_step(ctx, [sid], 1)[0] == 0
        ref = online_step(m, off, s_q)
        th = L.lrbms_get_field(ctx, sid, L.FIELD_THETA)
        assert np.abs(th @ P - m.mobility(s_q)).max() <= 1e-10 * np.abs(P).max()  # exact fit
        assert rel(th @ P, ref["theta"] @ P) < 1e-11
        assert rel(L.lrbms_get_field(ctx, sid, L.FIELD_P), ref["p"].reshape(-1, 3).T.reshape(-1)) < 1e-7
        assert rel(L.lrbms_get_field(ctx, sid, L.FIELD_S), ref["s"]) < 1e-7
    L.lrbms_destroy(ctx)
