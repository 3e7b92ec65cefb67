"""GPU parity of the high-dimensional scheme (Algorithm 1: SWIP-DG pressure of
Definition 1 with lambda(s^n), fluxes of Definition 2, upwind transport of
Definition 3) through lrbms_fine_step against the oracle's fine IMPES step.

The two sides solve the fine system differently (sparse LU in the oracle,
envelope Cholesky with one refinement step on the GPU), so the pressure
tolerance is max(1e-10, 10 x) the disagreement of two FP64 solvers of the
same system in the oracle (LU against dense Cholesky), computed per case."""
import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse.linalg as spla

from lrbms_cases import abi_offline, abi_problem, case, close_elementwise, rel
from oracle.swip import pressure_system
from test_gpu_parity import flux_tolerance

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1405_2810_gb300 import build, lrbms
    build.build()
    return lrbms


def _floor(m, s):
    lam = m.mobility(s)
    K, l = pressure_system(m.grid, m.perm, lam, m.c_pen, m.bc_type, m.p_D, m.v_N, swapped=m.swapped)
    x1 = spla.spsolve(K.tocsc(), l)
    x2 = sla.cho_solve(sla.cho_factor(K.toarray()), l)
    return float(np.linalg.norm(x1 - x2) / np.linalg.norm(x1))


CASES = [("small", dict(name="small")),
         ("ragged-tiles", dict(name="rect", kind="snapshots", n=(72, 40), S=(6, 4))),
         ("paper-bc", dict(name="paper_bc"))]


@pytest.mark.parametrize("label,kw", CASES, ids=[c[0] for c in CASES])
def test_fine_step_matches_oracle(L, label, kw):
    """Three fine steps, each from the oracle's fine state: pressure, fluxes,
    time step and saturation."""
    c = case(**kw)
    prob, m, co, off = c
    ctx = L.lrbms_create(hbm_budget=1 << 30, max_slots=2)
    sid = L.lrbms_offline_load(ctx, abi_problem(prob, m), abi_offline(co, off))
    s = prob.s0.copy()
    for _ in range(4):
        s = m.step(s)["s"]
    for _ in range(3):
        ref = m.step(s)
        tol = max(1e-10, 10 * _floor(m, s))
        L.lrbms_set_saturation(ctx, sid, s)
        assert L.lrbms_fine_step(ctx, [sid], 1)[0] == 0
        p = L.lrbms_get_field(ctx, sid, L.FIELD_P)
        p_ref = ref["p"].reshape(-1, 3).T.reshape(-1)
        assert rel(p, p_ref) < tol and close_elementwise(p, p_ref, tol) <= tol
        tf = max(tol, flux_tolerance(c, ref) * tol / 1e-10)
        assert rel(L.lrbms_get_field(ctx, sid, L.FIELD_FLUX), ref["F"]) < tf
        assert rel(L.lrbms_get_field(ctx, sid, L.FIELD_DT), [ref["dt"]]) < tf
        s_gpu = L.lrbms_get_field(ctx, sid, L.FIELD_S)
        assert rel(s_gpu, ref["s"]) < tf and close_elementwise(s_gpu, ref["s"], tf) <= tf
        s = ref["s"]
    L.lrbms_destroy(ctx)


def test_fine_trajectory_mass_balance_and_bounds(L):
    """Ten fine steps of two simulations in one call: the water volume changes
    by the boundary outflow to FP64 round-off, 0 <= s <= 1 (T3, T4), and the
    saturation follows the oracle's fine trajectory."""
    prob, m, co, off = c = case("small")
    ctx = L.lrbms_create(hbm_budget=1 << 30, max_slots=4)
    ids = [L.lrbms_offline_load(ctx, abi_problem(prob, m), abi_offline(co, off)) for _ in range(2)]
    st = L.lrbms_fine_step(ctx, ids, 10)
    assert list(st) == [0, 0]
    s_ref, hist = m.run(prob.s0, 10)
    vol = prob.poro * m.grid.vol
    for sid in ids:
        s = np.empty(prob.n_cells)
        _t, out = L.lrbms_get_state(ctx, sid, s)
        assert abs((np.sum(vol * s) - np.sum(vol * prob.s0)) + out) <= 1e-13 * abs(out)
        assert s.min() >= -1e-14 and s.max() <= 1 + 1e-14
        assert rel(s, s_ref) < 1e-8
    L.lrbms_destroy(ctx)


def test_fine_step_rejects_fitted_velocity(L):
    prob, m, co, off = c = case("small")
    ctx = L.lrbms_create(hbm_budget=1 << 30, max_slots=2)
    sid = L.lrbms_offline_load(ctx, abi_problem(prob, m, velocity=1), abi_offline(co, off))
    with pytest.raises(L.LrbmsError) as ei:
        L.lrbms_fine_step(ctx, [sid], 1)
    assert ei.value.code == L.LRBMS_E_ARG
    L.lrbms_destroy(ctx)
