"""Mixed precision mode (FP32 components and bases for assembly and
reconstruction, FP32 factor with FP64 refinement) against the FP64 oracle.

Rounding the components to FP32 perturbs the assembled matrix by about
eps_32 relative, so the reduced solution carries an error of order
cond(A) eps_32; the flux of Definition 2 adds the cancellation of its penalty
term (sigma_max |p|_inf / rms(F)). Each step is started from the oracle's own
state, the per-field errors are reported, and they must stay within these
first-order rounding bounds (computed from the oracle's data); the mass
balance of the GPU trajectory is exact (the transport is FP64 in every
mode).

The target of 1e-5 relative on pressure and flux and 1e-6 absolute on
saturation is checked separately as a strict expected failure: FP32 storage
does not reach it (the paper's boundary conditions, "paper-bc", give the
largest errors and are the headline numbers), and an unexpected pass is
reported as a failure so that reaching the target shows up."""
import numpy as np
import pytest

from lrbms_cases import abi_offline, abi_problem, case, rel
from oracle.reduced import online_step

pytestmark = pytest.mark.gpu
EPS32 = float(np.finfo(np.float32).eps)


@pytest.fixture(scope="module")
def L():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1405_2810_gb300 import build, lrbms
    build.build()
    return lrbms


def _soa(p):
    return p.reshape(-1, 3).T.reshape(-1)


MIXED_CASES = [("small", dict(name="small")), ("small-snapshots", dict(name="small", kind="snapshots")),
               ("paper-bc", dict(name="paper_bc"))]
TARGET_P, TARGET_F, TARGET_S = 1e-5, 1e-5, 1e-6


def _worst_errors(L, kw, check=None):
    """Worst per-step (p rel, F rel, s abs) errors of the mixed mode over
    steps started from the oracle's states; check(k, case, ref, ep, ef, es,
    F_gpu) may assert per step."""
    c = case(**kw)
    prob, m, co, off = c
    ctx = L.lrbms_create(hbm_budget=1 << 30, max_slots=4, precision=L.LRBMS_MIXED,
                         solver=L.LRBMS_SOLVE_MIXED)
    sid = L.lrbms_offline_load(ctx, abi_problem(prob, m), abi_offline(co, off, False))
    s = prob.s0.copy()
    worst = np.zeros(3)
    for k in range(prob.n_steps):
        ref = online_step(m, off, s)
        if k % 10 == 0 or k == prob.n_steps - 1:
            L.lrbms_set_saturation(ctx, sid, s)
            assert L.lrbms_step(ctx, [sid], 1)[0] == 0
            ep = rel(L.lrbms_get_field(ctx, sid, L.FIELD_P), _soa(ref["p"]))
            ef = rel(L.lrbms_get_field(ctx, sid, L.FIELD_FLUX), ref["F"])
            s_gpu = L.lrbms_get_field(ctx, sid, L.FIELD_S)
            es = float(np.max(np.abs(s_gpu - ref["s"])))
            if check is not None:
                F_gpu = L.lrbms_get_field(ctx, sid, L.FIELD_FLUX)
                check(k, c, ref, ep, ef, es, F_gpu)
            worst = np.maximum(worst, [ep, ef, es])
        s = ref["s"]
    L.lrbms_destroy(ctx)
    return worst


@pytest.mark.parametrize("label,kw", MIXED_CASES, ids=[c[0] for c in MIXED_CASES])
def test_mixed_precision_field_errors_within_rounding_bounds(L, label, kw):
    def check(k, c, ref, ep, ef, es, F_gpu):
        prob, m, co, off = c
        cond = np.linalg.cond(ref["A"])
        cancel = off.c_pen * np.max(prob.perm) * np.abs(ref["p"]).max() / np.sqrt(np.mean(ref["F"] ** 2))
        bound_p = 50 * cond * EPS32
        assert ep <= bound_p, (k, ep, bound_p)
        assert ef <= bound_p * max(1.0, cancel), (k, ef, bound_p * cancel)
        # saturation: with uniform porosity the FP64 upwind update turns a
        # flux error into at most dt/(phi|e|) sum_f |dF_f| <= 4 cfl max|dF| /
        # (L_f max_e outflow_e), and the step dt (set by the largest outflow)
        # adds at most cfl max|dF| / (L_f max_e outflow_e); 8 leaves a margin
        g, F = m.grid, ref["F"]
        out = np.zeros(g.n_cells)  # sum of the positive outward fluxes per cell
        f = g.interior
        np.add.at(out, g.fe1[f], np.maximum(F[f], 0.0))
        np.add.at(out, g.fe2[f], np.maximum(-F[f], 0.0))
        np.add.at(out, g.bcell, np.maximum(F[g.bface] * g.bsign, 0.0))
        dF = np.abs(F_gpu - ref["F"]).max()
        bound_s = 8.0 * m.cfl * dF / (m.Lf * out.max()) + 1e-14
        assert es <= bound_s, (k, es, bound_s)

    worst = _worst_errors(L, kw, check)
    print(f"{label}: mixed-precision worst per-step errors: p {worst[0]:.2e} (rel), "
          f"F {worst[1]:.2e} (rel), s {worst[2]:.2e} (abs)")


@pytest.mark.xfail(strict=True, reason="FP32 storage of bases and components misses the mixed-mode target")
@pytest.mark.parametrize("label,kw", MIXED_CASES, ids=[c[0] for c in MIXED_CASES])
def test_mixed_precision_meets_target(L, label, kw):
    worst = _worst_errors(L, kw)
    assert worst[0] <= TARGET_P and worst[1] <= TARGET_F and worst[2] <= TARGET_S, worst


def test_mixed_precision_mass_balance(L):
    prob, m, co, off = c = case("small")
    ctx = L.lrbms_create(hbm_budget=1 << 30, max_slots=4, precision=L.LRBMS_MIXED,
                         solver=L.LRBMS_SOLVE_MIXED)
    sid = L.lrbms_offline_load(ctx, abi_problem(prob, m), abi_offline(co, off, False))
    assert L.lrbms_step(ctx, [sid], prob.n_steps)[0] == 0
    s = np.empty(prob.n_cells)
    _t, out = L.lrbms_get_state(ctx, sid, s)
    vol = prob.poro * m.grid.vol
    assert abs((np.sum(vol * s) - np.sum(vol * prob.s0)) + out) <= 1e-13 * abs(out)
    L.lrbms_destroy(ctx)
