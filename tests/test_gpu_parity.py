"""GPU parity: the CUDA online step through the C ABI against the FP64 oracle
(Algorithm 3, step 5). FP64 mode tolerance: 1e-10 relative per field."""
import numpy as np
import pytest

from lrbms_cases import abi_offline, abi_problem, a_blocks, case, rel
from oracle.reduced import online_step

pytestmark = pytest.mark.gpu
TOL = 1e-10


@pytest.fixture(scope="module")
def L():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1405_2810_gb300 import build, lrbms
    build.build()
    return lrbms


def _ctx(L, **kw):
    kw.setdefault("hbm_budget", 1 << 30)
    kw.setdefault("max_slots", 16)
    return L.lrbms_create(**kw)


def _load(L, ctx, c, s0=None, dense=False, **pkw):
    prob, m, co, off = c
    return L.lrbms_offline_load(ctx, abi_problem(prob, m, s0=s0, **pkw), abi_offline(co, off, dense))


def _soa(p):
    return p.reshape(-1, 3).T.reshape(-1)


def flux_tolerance(c, ref):
    """Relative flux tolerance: 1e-10, or the round-off floor of Definition 2
    when the penalty term sigma_f [p] cancels many digits (a large pressure
    level with a small pressure drop): 50 eps sigma_max |p|_inf / rms(F),
    computed from the oracle's own data."""
    prob, m, co, off = c
    sig_max = off.c_pen * np.max(prob.perm)
    scale = sig_max * np.abs(ref["p"]).max() / max(np.sqrt(np.mean(ref["F"] ** 2)), 1e-300)
    return max(TOL, 50 * np.finfo(float).eps * scale)


def _compare_step(L, ctx, sid, c, s, ref=None):
    prob, m, co, off = c
    if ref is None:
        ref = online_step(m, off, s)
    th = L.lrbms_get_field(ctx, sid, L.FIELD_THETA)
    assert rel(th @ off.P, ref["theta"] @ off.P) < TOL
    assert rel(L.lrbms_get_field(ctx, sid, L.FIELD_A), a_blocks(co, off, ref["A"])) < TOL
    assert rel(L.lrbms_get_field(ctx, sid, L.FIELD_RHS), ref["rhs"]) < TOL
    assert rel(L.lrbms_get_field(ctx, sid, L.FIELD_X), ref["x"]) < TOL
    assert rel(L.lrbms_get_field(ctx, sid, L.FIELD_P), _soa(ref["p"])) < TOL
    tf = flux_tolerance(c, ref)
    assert rel(L.lrbms_get_field(ctx, sid, L.FIELD_FLUX), ref["F"]) < tf
    assert rel(L.lrbms_get_field(ctx, sid, L.FIELD_DT), [ref["dt"]]) < tf
    assert rel(L.lrbms_get_field(ctx, sid, L.FIELD_S), ref["s"]) < tf
    return ref


SOLVERS = [0, 1]  # FP64 block Cholesky; FP32 block Cholesky with FP64 refinement


@pytest.mark.parametrize("solver", SOLVERS, ids=["fp64-solve", "mixed-solve"])
def test_single_step_every_field(L, solver):
    c = case("small")
    ctx = _ctx(L, solver=solver)
    sid = _load(L, ctx, c)
    st = L.lrbms_step(ctx, [sid], 1)
    assert st[0] == 0
    _compare_step(L, ctx, sid, c, c[0].s0)
    L.lrbms_destroy(ctx)


@pytest.mark.parametrize("solver", SOLVERS, ids=["fp64-solve", "mixed-solve"])
def test_trajectory_and_mass_balance(L, solver):
    """Whole 50-step trajectory of the 32x32 / 4x4 case; the cumulative
    boundary outflow equals the loss of water volume to FP64 round-off."""
    prob, m, co, off = c = case("small")
    ctx = _ctx(L, solver=solver)
    sid = _load(L, ctx, c)
    s = prob.s0.copy()
    t = 0.0
    out = 0.0
    for k in range(prob.n_steps):
        r = online_step(m, off, s)
        s = r["s"]
        t += r["dt"]
        out += r["dt"] * r["boundary_outflow"]
    st = L.lrbms_step(ctx, [sid], prob.n_steps)
    assert st[0] == 0
    s_gpu = np.empty(prob.n_cells)
    tg, mg = L.lrbms_get_state(ctx, sid, s_gpu)
    assert rel(s_gpu, s) < TOL
    assert abs(tg - t) <= TOL * t
    assert abs(mg - out) <= TOL * abs(out)
    vol = prob.poro * m.grid.vol
    assert abs((np.sum(vol * s_gpu) - np.sum(vol * prob.s0)) + mg) <= 1e-13 * abs(mg)
    L.lrbms_destroy(ctx)


def test_step_from_oracle_state(L):
    """One GPU step from the oracle's state after 20 steps (isolates per-step
    parity from trajectory drift)."""
    prob, m, co, off = c = case("small")
    s = prob.s0.copy()
    for _ in range(20):
        s = online_step(m, off, s)["s"]
    ctx = _ctx(L)
    sid = _load(L, ctx, c)
    L.lrbms_set_saturation(ctx, sid, s)
    assert L.lrbms_step(ctx, [sid], 1)[0] == 0
    _compare_step(L, ctx, sid, c, s)
    L.lrbms_destroy(ctx)


CASES = [
    ("small-snapshots", dict(name="small", kind="snapshots")),
    ("paper-bc", dict(name="paper_bc")),
    ("paper-bc-level-0", dict(name="paper_bc", p_inflow=0.0)),
    ("ragged-tiles", dict(name="rect", kind="snapshots", n=(72, 40), S=(6, 4))),
    ("one-subdomain", dict(name="rect", kind="snapshots", n=(16, 12), S=(1, 1))),
    ("column-of-subdomains", dict(name="rect", kind="snapshots", n=(12, 40), S=(1, 5))),
    ("strip", dict(name="strip", kind="snapshots", n=64, S=4)),
    ("swapped-weights", dict(name="small", kind="snapshots", swapped=True)),
]


@pytest.mark.parametrize("solver", SOLVERS, ids=["fp64-solve", "mixed-solve"])
@pytest.mark.parametrize("label,kw", CASES, ids=[c[0] for c in CASES])
def test_cases_three_steps(L, label, kw, solver):
    """Three steps, each started from the oracle's own state (so every
    step is compared on identical inputs)."""
    c = case(**kw)
    prob, m, co, off = c
    ctx = _ctx(L, solver=solver)
    sid = _load(L, ctx, c)
    s = prob.s0.copy()
    for _ in range(3):
        L.lrbms_set_saturation(ctx, sid, s)
        assert L.lrbms_step(ctx, [sid], 1)[0] == 0
        ref = _compare_step(L, ctx, sid, c, s)
        s = ref["s"]
    L.lrbms_destroy(ctx)


def test_dense_profiles_and_fixed_dt(L):
    prob, m, co, off = c = case("small")
    ctx = _ctx(L)
    sid = _load(L, ctx, c, dense=True, dt_mode=1, dt_fixed=1e-3)
    s = prob.s0.copy()
    m.dt_fixed = 1e-3
    try:
        for _ in range(2):
            assert L.lrbms_step(ctx, [sid], 1)[0] == 0
            s = _compare_step(L, ctx, sid, c, s)["s"]
    finally:
        m.dt_fixed = None
    L.lrbms_destroy(ctx)


@pytest.mark.parametrize("solver", SOLVERS, ids=["fp64-solve", "mixed-solve"])
def test_batch_equals_alone_bitwise(L, solver):
    """Simulations of different shapes and basis sizes stepped in one launch
    give bitwise the same results as each stepped alone."""
    cs = [case("small"), case("rect", kind="snapshots", n=(72, 40), S=(6, 4)),
          case("paper_bc", p_inflow=0.0), case("small", kind="snapshots")]
    ctx = _ctx(L, solver=solver)
    ids = [_load(L, ctx, c) for c in cs]
    st = L.lrbms_step(ctx, ids, 5)
    assert list(st) == [0] * len(cs)
    mixed = [L.lrbms_get_field(ctx, i, L.FIELD_S) for i in ids]
    L.lrbms_destroy(ctx)
    for c, sm in zip(cs, mixed):
        ctx = _ctx(L, solver=solver)
        sid = _load(L, ctx, c)
        assert L.lrbms_step(ctx, [sid], 5)[0] == 0
        alone = L.lrbms_get_field(ctx, sid, L.FIELD_S)
        assert np.array_equal(alone, sm)
        L.lrbms_destroy(ctx)


def test_failed_simulation_is_isolated(L):
    """A corrupt offline blob (host-side fault injection: a negated diagonal
    block makes the reduced matrix indefinite) and a NaN saturation freeze
    only their own simulations; the others match the clean run bitwise."""
    good = case("small")
    prob, m, co, off = good
    ctx = _ctx(L)
    clean = _load(L, ctx, good)
    bad_off = abi_offline(co, off)
    bad_off["Dblk"] = bad_off["Dblk"].copy()
    n0 = off.N_E[0]
    bad_off["Dblk"][: n0 * n0] *= -1.0  # c block of subdomain 0
    bad_off["Dblk"][n0 * n0: (off.M + 1) * n0 * n0] *= -1.0
    bad = L.lrbms_offline_load(ctx, abi_problem(prob, m), bad_off)
    s_nan = prob.s0.copy()
    s_nan[7] = np.nan
    nan_id = _load(L, ctx, good, s0=s_nan)
    st = L.lrbms_step(ctx, [clean, bad, nan_id], 3)
    assert st[0] == L.LRBMS_OK
    assert st[1] == L.LRBMS_E_NOT_SPD
    assert st[2] in (L.LRBMS_E_NONFINITE, L.LRBMS_E_NOT_SPD)
    s_clean = L.lrbms_get_field(ctx, clean, L.FIELD_S)
    L.lrbms_destroy(ctx)
    ctx = _ctx(L)
    ref = _load(L, ctx, good)
    L.lrbms_step(ctx, [ref], 3)
    assert np.array_equal(L.lrbms_get_field(ctx, ref, L.FIELD_S), s_clean)
    L.lrbms_destroy(ctx)


def test_budget_admission_and_slot_reuse(L):
    c = case("small")
    ctx = _ctx(L, hbm_budget=3 << 20, max_slots=8)
    ids = []
    with pytest.raises(L.LrbmsError) as ei:
        for _ in range(8):
            ids.append(_load(L, ctx, c))
    assert ei.value.code == L.LRBMS_E_BUDGET
    assert len(ids) >= 1
    used, cap = L.lrbms_memory(ctx)
    assert used <= cap
    L.lrbms_release(ctx, ids[0])
    again = _load(L, ctx, c)
    assert L.lrbms_step(ctx, [again], 2)[0] == 0
    L.lrbms_destroy(ctx)


def test_run_returns_last_step_fields(L):
    """lrbms_run (n steps, then the saturation, pressure and fluxes of the
    last step into caller buffers) against the oracle's trajectory."""
    prob, m, co, off = c = case("small")
    ctx = _ctx(L, solver=1)
    sid = _load(L, ctx, c)
    s = prob.s0.copy()
    for _ in range(4):
        ref = online_step(m, off, s)
        s = ref["s"]
    s_out = np.empty(prob.n_cells)
    p_out = np.empty(3 * prob.n_cells)
    F_out = np.empty(m.grid.n_faces)
    L.lrbms_run(ctx, sid, 4, s_out, p_out, F_out)
    assert rel(s_out, s) < TOL
    assert rel(p_out, _soa(ref["p"])) < TOL
    assert rel(F_out, ref["F"]) < flux_tolerance(c, ref)
    L.lrbms_destroy(ctx)


def test_fixed_step_beyond_cfl_bound_is_refused(L):
    """A fixed time step twice the CFL bound with CFL number 1 (reading R12
    with cfl = 1, from the oracle's fluxes) freezes the simulation with
    LRBMS_E_CFL and leaves its saturation unchanged; half the bound steps
    normally and matches the oracle."""
    from oracle.transport import cfl_dt
    prob, m, co, off = c = case("small")
    ref = online_step(m, off, prob.s0)
    bound = cfl_dt(m.grid, ref["F"], m.poro, m.Lf, 1.0)
    ctx = _ctx(L)
    big = _load(L, ctx, c, dt_mode=1, dt_fixed=2.0 * bound)
    ok = _load(L, ctx, c, dt_mode=1, dt_fixed=0.5 * bound)
    st = L.lrbms_step(ctx, [big, ok], 1)
    assert st[0] == L.LRBMS_E_CFL and st[1] == 0
    assert np.array_equal(L.lrbms_get_field(ctx, big, L.FIELD_S), prob.s0)
    m.dt_fixed = 0.5 * bound
    try:
        _compare_step(L, ctx, ok, c, prob.s0)
    finally:
        m.dt_fixed = None
    L.lrbms_destroy(ctx)


@pytest.mark.parametrize("solver", SOLVERS, ids=["fp64-solve", "mixed-solve"])
def test_graph_replay_equals_direct_launches(L, solver):
    """Steps replayed from the captured CUDA graph give bitwise the results of
    the same steps launched kernel by kernel (profiled steps are launched
    directly), and the launch count grows by the kernels of each step."""
    c = case("small", kind="snapshots")
    out = []
    for profiled in (False, True):
        ctx = _ctx(L, solver=solver)
        sid = _load(L, ctx, c)
        if profiled:
            L.lrbms_profile_start(ctx, 6)
        n0 = L.lrbms_launch_count(ctx)
        assert L.lrbms_step(ctx, [sid], 6)[0] == 0
        per_step = (L.lrbms_launch_count(ctx) - n0) / 6
        if profiled:
            ph, st = L.lrbms_profile_read(ctx, 6)
            assert len(st) == 6 and np.all(ph >= 0)
        out.append((L.lrbms_get_field(ctx, sid, L.FIELD_S), L.lrbms_get_field(ctx, sid, L.FIELD_X), per_step))
        L.lrbms_destroy(ctx)
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])
    assert out[0][2] == out[1][2] >= 7


@pytest.mark.parametrize("dense", [False, True], ids=["threshold-profiles", "dense-profiles"])
def test_fitted_velocity_variant(L, dense):
    """Fluxes with the fitted mobility sum_q theta_q Lambda^q (reading R7's
    variant) against the oracle's variant, three steps from its states."""
    prob, m, co, off = c = case("small", kind="snapshots")
    ctx = _ctx(L, solver=1)
    sid = _load(L, ctx, c, dense=dense, velocity=1)
    s = prob.s0.copy()
    for _ in range(8):
        s = online_step(m, off, s, velocity="fitted")["s"]
    for _ in range(3):
        L.lrbms_set_saturation(ctx, sid, s)
        assert L.lrbms_step(ctx, [sid], 1)[0] == 0
        ref = online_step(m, off, s, velocity="fitted")
        _compare_step(L, ctx, sid, c, s, ref=ref)
        s = ref["s"]
    L.lrbms_destroy(ctx)


@pytest.mark.parametrize("solver", SOLVERS, ids=["fp64-solve", "mixed-solve"])
def test_bounded_wait_timeout_is_isolated(L, solver):
    """Failure detection without a GPU fault: one simulation's solve withholds
    a bulk copy (test hook), its bounded wait runs out after about 2 s, and it
    stops with LRBMS_E_TIMEOUT; the other simulations of the same launches
    give bitwise the results of a clean run, and the context stays usable."""
    c = case("small", kind="snapshots")
    ctx = _ctx(L, solver=solver)
    ids = [_load(L, ctx, c) for _ in range(3)]
    assert list(L.lrbms_step(ctx, ids, 2)) == [0, 0, 0]
    L.lrbms_test_withhold_copy(ctx, ids[1])
    st = L.lrbms_step(ctx, ids, 3)
    assert list(st) == [0, L.LRBMS_E_TIMEOUT, 0]
    got = [L.lrbms_get_field(ctx, i, L.FIELD_S) for i in (ids[0], ids[2])]
    L.lrbms_destroy(ctx)
    ctx = _ctx(L, solver=solver)
    ref = _load(L, ctx, c)
    assert L.lrbms_step(ctx, [ref], 5)[0] == 0
    want = L.lrbms_get_field(ctx, ref, L.FIELD_S)
    L.lrbms_destroy(ctx)
    assert np.array_equal(got[0], want) and np.array_equal(got[1], want)


def test_autotuned_sizes_do_not_change_results(L):
    """The autotuner's choice of CTA sizes for assembly and reconstruction is
    recorded per shape class, and a context forced through every candidate
    size (by stepping simulations of several classes) still matches the
    oracle; a second context gives bitwise the same saturation."""
    c = case("small", kind="snapshots")
    out = []
    for _ in range(2):
        ctx = _ctx(L, solver=1)
        sid = _load(L, ctx, c)
        with pytest.raises(L.LrbmsError):
            L.lrbms_tuned_threads(ctx, [sid])
        assert L.lrbms_step(ctx, [sid], 3)[0] == 0
        ta, tr = L.lrbms_tuned_threads(ctx, [sid])
        assert ta in (64, 128, 256, 512) and tr in (128, 256, 512, 1024)
        out.append(L.lrbms_get_field(ctx, sid, L.FIELD_S))
        L.lrbms_destroy(ctx)
    assert np.array_equal(out[0], out[1])
