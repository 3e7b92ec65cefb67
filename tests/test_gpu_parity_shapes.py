"""GPU parity at the shapes the batched bench and the serving pool run
(Algorithm 3, step 5; Eq. reducedSystem): 8x8 subdomains with basis sizes
from U{5..30}, 8x8 subdomains with sizes 17, 24, 30 and 32 side by side, and
16x16 subdomains (17 blocks per envelope row). Every field of a step is
compared with the FP64 oracle both in relative L2 norm and element by
element (max |gpu - oracle| / max |oracle|), from the oracle's own states,
for both reduced solvers."""
import numpy as np
import pytest

from lrbms_cases import SHAPES, abi_offline, abi_problem, a_blocks, close_elementwise, rel, shape_case, shape_states
from oracle.reduced import online_step
from test_gpu_parity import flux_tolerance

pytestmark = pytest.mark.gpu
TOL = 1e-10
LATE = 12  # oracle step whose state starts the second compared step


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


def _check_fields(L, ctx, sid, c, s):
    """Every field of the last step against the oracle's step from s."""
    prob, m, co, off = c
    ref = online_step(m, off, s)
    tf = flux_tolerance(c, ref)
    pairs = [
        ("fitted mobility", L.lrbms_get_field(ctx, sid, L.FIELD_THETA) @ off.P, ref["theta"] @ off.P, TOL),
        ("A", L.lrbms_get_field(ctx, sid, L.FIELD_A), a_blocks(co, off, ref["A"]), TOL),
        ("rhs", L.lrbms_get_field(ctx, sid, L.FIELD_RHS), ref["rhs"], TOL),
        ("x", L.lrbms_get_field(ctx, sid, L.FIELD_X), ref["x"], TOL),
        ("p", L.lrbms_get_field(ctx, sid, L.FIELD_P), _soa(ref["p"]), TOL),
        ("F", L.lrbms_get_field(ctx, sid, L.FIELD_FLUX), ref["F"], tf),
        ("dt", L.lrbms_get_field(ctx, sid, L.FIELD_DT), np.array([ref["dt"]]), tf),
        ("s", L.lrbms_get_field(ctx, sid, L.FIELD_S), ref["s"], tf),
    ]
    for name, got, want, tol in pairs:
        r2, re = rel(got, want), close_elementwise(got, want, tol)
        assert r2 <= tol, (name, "L2", r2, tol)
        assert re <= tol, (name, "element-wise", re, tol)


@pytest.mark.parametrize("solver", [0, 1], ids=["fp64-solve", "mixed-solve"])
@pytest.mark.parametrize("label", list(SHAPES))
def test_bench_shape_steps(L, label, solver):
    """One step from s^0 and one from the oracle's state after LATE steps."""
    c = shape_case(label)
    prob, m, co, off = c
    states = shape_states(label, LATE)
    ctx = L.lrbms_create(hbm_budget=1 << 30, max_slots=2, solver=solver)
    sid = L.lrbms_offline_load(ctx, abi_problem(prob, m), abi_offline(co, off))
    for s in (states[0], states[LATE]):
        L.lrbms_set_saturation(ctx, sid, s)
        assert L.lrbms_step(ctx, [sid], 1)[0] == 0
        _check_fields(L, ctx, sid, c, s)
    L.lrbms_destroy(ctx)


@pytest.mark.parametrize("solver", [0, 1], ids=["fp64-solve", "mixed-solve"])
def test_bench_shapes_in_one_launch(L, solver):
    """All shapes stepped together (one launch per phase, the launch shape
    set by the largest system), two unrotated copies each; every
    simulation still matches the oracle field by field."""
    ctx = L.lrbms_create(hbm_budget=2 << 30, max_slots=8, solver=solver)
    sims = []
    for label in SHAPES:
        c = shape_case(label)
        prob, m, co, off = c
        s = shape_states(label, LATE)[LATE]
        for _ in range(2):
            sid = L.lrbms_offline_load(ctx, abi_problem(prob, m), abi_offline(co, off))
            L.lrbms_set_saturation(ctx, sid, s)
            sims.append((sid, c, s))
    st = L.lrbms_step(ctx, [sid for sid, _, _ in sims], 1)
    assert list(st) == [0] * len(sims)
    for sid, c, s in sims:
        _check_fields(L, ctx, sid, c, s)
    L.lrbms_destroy(ctx)


def test_bench_shape_trajectory_mass_balance(L):
    """LATE steps of the 8x8 bench shape with the mixed solver: the saturation
    matches the oracle's trajectory, and the water volume changes by the
    cumulative boundary outflow to FP64 round-off."""
    c = shape_case("bench-8x8")
    prob, m, co, off = c
    ctx = L.lrbms_create(hbm_budget=1 << 30, max_slots=2, solver=1)
    sid = L.lrbms_offline_load(ctx, abi_problem(prob, m), abi_offline(co, off))
    assert L.lrbms_step(ctx, [sid], LATE)[0] == 0
    s_gpu = np.empty(prob.n_cells)
    _, mg = L.lrbms_get_state(ctx, sid, s_gpu)
    s_ref = shape_states("bench-8x8", LATE)[LATE]
    assert rel(s_gpu, s_ref) < TOL and close_elementwise(s_gpu, s_ref, TOL) <= TOL
    vol = prob.poro * m.grid.vol
    assert abs((np.sum(vol * s_gpu) - np.sum(vol * prob.s0)) + mg) <= 1e-13 * abs(mg)
    info = L.lrbms_get_field(ctx, sid, L.FIELD_SOLVE_INFO, dtype=np.int32)
    assert info[5] == LATE  # one reduced solve per step
    assert 1 <= info[2] < LATE  # the FP32 factor was reused on some steps
    L.lrbms_destroy(ctx)


@pytest.mark.parametrize("label", ["bench-8x8", "serve-16x16"])
def test_staged_refactorisation(L, label):
    """Mixed solver with the next FP32 factor built over 4 steps (period 4):
    the whole first factor at step 0, staged builds completing at steps 4
    and 8. Every solve is a warm conjugate-gradient solve (no stale retry,
    no FP64 redo), the result is the same bitwise with another simulation
    in the batch, and a further step from the oracle's state (with the
    staged factor of step 8 as preconditioner) matches the oracle in every
    field, element by element. On the bench shape the LATE-step trajectory
    also matches the oracle's, with the mass balance."""
    c = shape_case(label)
    prob, m, co, off = c
    other = shape_case("bench-8x8-wide")
    out = []
    for batch in (False, True):
        ctx = L.lrbms_create(hbm_budget=2 << 30, max_slots=4, solver=1, refactor_period=4, refactor_stages=4)
        sid = L.lrbms_offline_load(ctx, abi_problem(prob, m), abi_offline(co, off))
        ids = [sid]
        if batch:
            ids.append(L.lrbms_offline_load(ctx, abi_problem(other[0], other[1]), abi_offline(other[2], other[3])))
        assert list(L.lrbms_step(ctx, ids, LATE)) == [0] * len(ids)
        s_gpu = np.empty(prob.n_cells)
        _, mg = L.lrbms_get_state(ctx, sid, s_gpu)
        info = L.lrbms_get_field(ctx, sid, L.FIELD_SOLVE_INFO, dtype=np.int32)
        out.append((s_gpu, mg, info))
        if not batch:
            s = shape_states(label, LATE)[LATE]
            L.lrbms_set_saturation(ctx, sid, s)
            assert L.lrbms_step(ctx, [sid], 1)[0] == 0
            _check_fields(L, ctx, sid, c, s)
        L.lrbms_destroy(ctx)
    (s_gpu, mg, info), (s_b, mg_b, info_b) = out
    assert info[5] == LATE and info[2] == 3 and info[1] == 0 and info[3] == 0, info
    assert np.array_equal(s_gpu, s_b) and mg == mg_b and np.array_equal(info, info_b)
    if label == "bench-8x8":
        s_ref = shape_states(label, LATE)[LATE]
        assert rel(s_gpu, s_ref) < TOL and close_elementwise(s_gpu, s_ref, TOL) <= TOL
        vol = prob.poro * m.grid.vol
        assert abs((np.sum(vol * s_gpu) - np.sum(vol * prob.s0)) + mg) <= 1e-13 * abs(mg)


@pytest.mark.parametrize("stages", [1, 4])
def test_warm_admission_is_bitwise_a_cold_start(L, stages):
    """Unrotated clones of a resting simulation start with its FP32 factor
    (computed once for the source): the source, two clones and a cold load
    of the same data give bitwise the same states, solutions and solver
    counters over LATE steps; a source whose saturation was set afresh drops
    the precomputed factor and again matches a cold load."""
    c = shape_case("bench-8x8")
    prob, m, co, off = c
    ctx = L.lrbms_create(hbm_budget=2 << 30, max_slots=8, solver=1, refactor_period=4, refactor_stages=stages)
    src = L.lrbms_offline_load(ctx, abi_problem(prob, m), abi_offline(co, off))
    warm = [L.lrbms_clone(ctx, src, None), L.lrbms_clone(ctx, src, None)]
    cold = L.lrbms_offline_load(ctx, abi_problem(prob, m), abi_offline(co, off))
    info0 = [L.lrbms_get_field(ctx, i, L.FIELD_SOLVE_INFO, dtype=np.int32) for i in (src, *warm, cold)]
    assert [int(v[2]) for v in info0] == [1, 1, 1, 0]  # factors held before any step
    other = L.lrbms_offline_load(ctx, abi_problem(prob, m), abi_offline(co, off))
    moved = L.lrbms_clone(ctx, other, None)
    s_late = shape_states("bench-8x8", LATE)[LATE]
    L.lrbms_set_saturation(ctx, other, s_late)  # drops other's factor
    cold_late = L.lrbms_offline_load(ctx, abi_problem(prob, m), abi_offline(co, off))
    L.lrbms_set_saturation(ctx, cold_late, s_late)
    ids = [src, *warm, cold, other, cold_late, moved]
    assert list(L.lrbms_step(ctx, ids, LATE)) == [0] * len(ids)
    fields = {i: (L.lrbms_get_field(ctx, i, L.FIELD_S), L.lrbms_get_field(ctx, i, L.FIELD_X),
                  L.lrbms_get_field(ctx, i, L.FIELD_SOLVE_INFO, dtype=np.int32)) for i in ids}
    for i in (src, *warm, moved):
        for a, b in zip(fields[i], fields[cold]):
            assert np.array_equal(a, b), i
    for a, b in zip(fields[other], fields[cold_late]):
        assert np.array_equal(a, b)
    L.lrbms_destroy(ctx)
