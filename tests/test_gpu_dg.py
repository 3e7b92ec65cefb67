"""GPU parity of the piecewise-linear DG saturation with the slope limiter
(Definition 3 with k = 1; Section 3.4, Eq. limiterMain) against the oracle:
the reduced online step (Algorithm 3, step 5) and the high-dimensional step
(Algorithm 1), each started from the oracle's own state (means and slopes),
and whole trajectories with exact mass balance."""
import numpy as np
import pytest

from lrbms_cases import abi_offline, abi_problem, case, close_elementwise, rel
from oracle.reduced import online_step_dg
from oracle.transport_dg import fine_step_dg
from test_gpu_fine_step import _floor
from test_gpu_parity import flux_tolerance

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


def _set_state(L, ctx, sid, c):
    L.lrbms_set_saturation(ctx, sid, np.ascontiguousarray(c[:, 0]))
    L.lrbms_set_slopes(ctx, sid, np.ascontiguousarray(c[:, 1:].T.reshape(-1)))


def _get_state(L, ctx, sid, n):
    s = L.lrbms_get_field(ctx, sid, L.FIELD_S)
    sl = L.lrbms_get_field(ctx, sid, L.FIELD_SLOPES).reshape(2, n)
    return np.column_stack([s, sl[0], sl[1]])


def _check(got, want, tol, what):
    assert rel(got, want) <= tol, (what, rel(got, want), tol)
    assert close_elementwise(got, want, tol) <= tol, (what, close_elementwise(got, want, tol), tol)


@pytest.mark.parametrize("solver", [0, 1], ids=["fp64-solve", "mixed-solve"])
@pytest.mark.parametrize("kw", [dict(name="small"), dict(name="rect", kind="snapshots", n=(72, 40), S=(6, 4))],
                         ids=["small", "ragged-tiles"])
def test_reduced_dg_steps_from_oracle_states(L, kw, solver):
    prob, m, co, off = c = case(**kw)
    ctx = L.lrbms_create(hbm_budget=1 << 30, max_slots=2, solver=solver)
    sid = L.lrbms_offline_load(ctx, abi_problem(prob, m, transport=1), abi_offline(co, off))
    st = np.zeros((prob.n_cells, 3))
    for _ in range(6):
        st = online_step_dg(m, off, st)["c"]
    for _ in range(3):
        ref = online_step_dg(m, off, st)
        _set_state(L, ctx, sid, st)
        assert L.lrbms_step(ctx, [sid], 1)[0] == 0
        tf = flux_tolerance(c, dict(p=ref["p"], F=ref["F"]))
        _check(L.lrbms_get_field(ctx, sid, L.FIELD_X), ref["x"], TOL, "x")
        _check(L.lrbms_get_field(ctx, sid, L.FIELD_FLUX), ref["F"], tf, "F")
        _check(L.lrbms_get_field(ctx, sid, L.FIELD_DT), np.array([ref["dt"]]), tf, "dt")
        got = _get_state(L, ctx, sid, prob.n_cells)
        _check(got[:, 0], ref["c"][:, 0], tf, "means")
        _check(got[:, 1:], ref["c"][:, 1:], tf, "slopes")
        st = ref["c"]
    L.lrbms_destroy(ctx)


def test_reduced_dg_trajectory_mass_balance(L):
    """Twelve DG steps from s0: the state follows the oracle's trajectory and
    the water volume changes by the boundary outflow to FP64 round-off."""
    prob, m, co, off = c = case("small")
    ctx = L.lrbms_create(hbm_budget=1 << 30, max_slots=2, solver=1)
    sid = L.lrbms_offline_load(ctx, abi_problem(prob, m, transport=1), abi_offline(co, off))
    assert L.lrbms_step(ctx, [sid], 12)[0] == 0
    st = np.zeros((prob.n_cells, 3))
    for _ in range(12):
        st = online_step_dg(m, off, st)["c"]
    got = _get_state(L, ctx, sid, prob.n_cells)
    assert rel(got, st) < 1e-8
    _t, out = L.lrbms_get_state(ctx, sid, None)
    vol = prob.poro * m.grid.vol
    assert abs(np.sum(vol * got[:, 0]) + out) <= 1e-13 * abs(out)
    L.lrbms_destroy(ctx)


def test_fine_dg_step_matches_oracle(L):
    """Algorithm 1 with the DG saturation and the limiter (lrbms_fine_step)."""
    prob, m, co, off = c = case("small")
    ctx = L.lrbms_create(hbm_budget=1 << 30, max_slots=2)
    sid = L.lrbms_offline_load(ctx, abi_problem(prob, m, transport=1), abi_offline(co, off))
    st = np.zeros((prob.n_cells, 3))
    for _ in range(5):
        st = fine_step_dg(m, st)["c"]
    for _ in range(2):
        ref = fine_step_dg(m, st)
        tol = max(TOL, 10 * _floor(m, st[:, 0]))
        _set_state(L, ctx, sid, st)
        assert L.lrbms_fine_step(ctx, [sid], 1)[0] == 0
        tf = max(tol, flux_tolerance(c, dict(p=ref["p"], F=ref["F"])) * tol / TOL)
        _check(L.lrbms_get_field(ctx, sid, L.FIELD_FLUX), ref["F"], tf, "F")
        got = _get_state(L, ctx, sid, prob.n_cells)
        _check(got, ref["c"], tf, "state")
        st = ref["c"]
    L.lrbms_destroy(ctx)


def test_fv_and_dg_simulations_in_one_batch(L):
    """A finite-volume and a DG simulation stepped together give bitwise the
    results of each stepped alone."""
    prob, m, co, off = c = case("small", kind="snapshots")
    out = {}
    for mode in ("batch", "alone"):
        if mode == "batch":
            ctx = L.lrbms_create(hbm_budget=1 << 30, max_slots=4, solver=1)
            ids = [L.lrbms_offline_load(ctx, abi_problem(prob, m, transport=t), abi_offline(co, off)) for t in (0, 1)]
            assert list(L.lrbms_step(ctx, ids, 4)) == [0, 0]
            out[mode] = [_get_state(L, ctx, i, prob.n_cells) for i in ids]
            L.lrbms_destroy(ctx)
        else:
            res = []
            for t in (0, 1):
                ctx = L.lrbms_create(hbm_budget=1 << 30, max_slots=2, solver=1)
                i = L.lrbms_offline_load(ctx, abi_problem(prob, m, transport=t), abi_offline(co, off))
                assert L.lrbms_step(ctx, [i], 4)[0] == 0
                res.append(_get_state(L, ctx, i, prob.n_cells))
                L.lrbms_destroy(ctx)
            out[mode] = res
    for a, b in zip(out["batch"], out["alone"]):
        assert np.array_equal(a, b)
