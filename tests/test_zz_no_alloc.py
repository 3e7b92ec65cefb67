"""The allocation-free reduced solve (lrbms_solve_noalloc).

The entry point exists for callers that cannot call cudaMalloc: a host
process whose device memory belongs to another allocator, or a time-critical
loop in which an allocation's implicit synchronisation or possible failure is
not allowed. Its working memory is one fixed array in device memory that all
calls share. The tests compare it with the solve inside lrbms_step and with
the oracle's dense FP64 solve, two calls in a row each (so leftover contents
of the shared array cannot leak into the next result), and check that every
size limit and argument check answers with its own status."""
import numpy as np
import pytest

from lrbms_cases import a_blocks, abi_offline, abi_problem, case, close_elementwise, rel, shape_case, shape_states
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


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


@pytest.mark.parametrize("solver", [0, 1], ids=["fp64-solve", "mixed-solve"])
def test_noalloc_solve_matches_step_twice(L, solver):
    import torch
    prob, m, co, off = c = case("small", kind="snapshots")
    ctx = L.lrbms_create(hbm_budget=256 << 20, max_slots=2, solver=solver)
    sid = L.lrbms_offline_load(ctx, abi_problem(prob, m), abi_offline(co, off))
    for call in range(2):  # a different system on each call (the state advances)
        assert L.lrbms_step(ctx, [sid], 1)[0] == 0
        A = _dev(L.lrbms_get_field(ctx, sid, L.FIELD_A))
        b = _dev(L.lrbms_get_field(ctx, sid, L.FIELD_RHS))
        x_ref = L.lrbms_get_field(ctx, sid, L.FIELD_X)
        x = torch.full_like(b, np.nan)
        rc = L.lrbms_solve_noalloc(prob.Sx, prob.Sy, off.N_E, A, b, x, solver=solver)
        assert rc == L.LRBMS_OK
        assert rel(x.cpu().numpy(), x_ref) < TOL, call
    L.lrbms_destroy(ctx)


@pytest.mark.parametrize("solver", [0, 1], ids=["fp64-solve", "mixed-solve"])
@pytest.mark.parametrize("label", ["bench-8x8", "bench-8x8-wide"])
def test_noalloc_solve_matches_oracle_at_bench_shapes(L, label, solver):
    """The oracle's assembled systems of two different steps (basis sizes
    up to 32) solved back to back: x against the oracle's dense Cholesky
    solve, in L2 and element by element."""
    import torch
    prob, m, co, off = shape_case(label)
    states = shape_states(label, 12)
    for s in (states[0], states[12]):
        ref = online_step(m, off, s)
        A = _dev(a_blocks(co, off, ref["A"]))
        b = _dev(ref["rhs"])
        x = torch.full_like(b, np.nan)
        assert L.lrbms_solve_noalloc(prob.Sx, prob.Sy, off.N_E, A, b, x, solver=solver) == L.LRBMS_OK
        got = x.cpu().numpy()
        assert rel(got, ref["x"]) < TOL and close_elementwise(got, ref["x"], TOL) <= TOL


def test_noalloc_mixed_falls_back_to_fp64_on_ill_conditioning(L):
    """A system shifted towards singularity (cond about 1e9, beyond what an
    FP32 factor can refine) makes the mixed solve fall back to the FP64
    factorisation inside the same kernel: its result equals the FP64 solve's,
    and both agree with the oracle's dense solve to the conditioning bound."""
    import scipy.linalg as sla
    import torch
    prob, m, co, off = shape_case("bench-8x8")
    ref = online_step(m, off, shape_states("bench-8x8", 12)[12])
    Ad = ref["A"]
    ev = sla.eigvalsh(Ad)
    As = Ad - (ev[0] - ev[-1] * 1e-9) * np.eye(len(ev))  # keeps the block pattern
    cond = ev[-1] / (ev[-1] * 1e-9)
    x_dense = sla.cho_solve(sla.cho_factor(As), ref["rhs"])
    A = _dev(a_blocks(co, off, As))
    b = _dev(ref["rhs"])
    outs = []
    for solver in (0, 1, 1):
        x = torch.full_like(b, np.nan)
        assert L.lrbms_solve_noalloc(prob.Sx, prob.Sy, off.N_E, A, b, x, solver=solver) == L.LRBMS_OK
        outs.append(x.cpu().numpy())
    assert np.array_equal(outs[1], outs[0]) and np.array_equal(outs[2], outs[0])
    assert rel(outs[0], x_dense) < 100 * cond * np.finfo(float).eps


def test_noalloc_argument_checks(L):
    """Host arrays, another dtype, a wrong size or a non-contiguous tensor
    are refused before any device work; so is a non-finite right-hand side
    after the solve (a NaN solution is not reported as converged)."""
    import torch
    prob, m, co, off = shape_case("bench-8x8")
    ref = online_step(m, off, prob.s0)
    A = _dev(a_blocks(co, off, ref["A"]))
    b = _dev(ref["rhs"])
    x = torch.zeros_like(b)
    S = (prob.Sx, prob.Sy, off.N_E)
    assert L.lrbms_solve_noalloc(*S, A.cpu().numpy(), b, x) == L.LRBMS_E_ARG
    assert L.lrbms_solve_noalloc(*S, A.float(), b, x) == L.LRBMS_E_ARG
    assert L.lrbms_solve_noalloc(*S, A[:-1], b, x) == L.LRBMS_E_ARG
    assert L.lrbms_solve_noalloc(*S, A, torch.zeros(2 * b.numel(), dtype=torch.float64, device="cuda")[::2],
                                 x) == L.LRBMS_E_ARG
    assert L.lrbms_solve_noalloc(*S, A, b, x.cpu()) == L.LRBMS_E_ARG
    # the library itself refuses a host pointer (the binding's checks bypassed)
    ne = np.ascontiguousarray(off.N_E, dtype=np.int32)
    host = np.zeros(A.numel())
    assert L.library().lrbms_solve_noalloc(prob.Sx, prob.Sy, ne.ctypes.data, host.ctypes.data, b.data_ptr(),
                                           x.data_ptr(), 0, 0, None) == L.LRBMS_E_ARG
    bn = b.clone()
    bn[5] = float("nan")
    for solver in (0, 1):
        assert L.lrbms_solve_noalloc(*S, A, bn, x, solver=solver) == L.LRBMS_E_NONFINITE
    # and the array is usable again right after
    assert L.lrbms_solve_noalloc(*S, A, b, x, solver=1) == L.LRBMS_OK
    assert rel(x.cpu().numpy(), ref["x"]) < TOL


def _zeros_for(L, Sx, Sy, NE):
    import torch
    na, n = L.noalloc_sizes(Sx, Sy, NE)
    return (torch.zeros(na, dtype=torch.float64, device="cuda"), torch.zeros(n, dtype=torch.float64, device="cuda"),
            torch.zeros(n, dtype=torch.float64, device="cuda"))


def test_noalloc_rejects_systems_beyond_its_limits(L):
    """Three different limits, each reached alone (all return
    LRBMS_E_BUDGET before any launch):
      - the 32 MiB array: 100 x 7 subdomains of 8 functions fit one CTA's
        shared memory but need about 34 MiB of factor panels;
      - shared memory: 16 x 16 subdomains of 32 functions need a panel row
        and work vectors beyond one CTA's shared memory;
      - the subdomain count of the host-side tables (at most 4096)."""
    for Sx, Sy, n in ((100, 7, 8), (16, 16, 32), (65, 65, 1)):
        NE = np.full(Sx * Sy, n, dtype=np.int32)
        A, b, x = _zeros_for(L, Sx, Sy, NE)
        assert L.lrbms_solve_noalloc(Sx, Sy, NE, A, b, x) == L.LRBMS_E_BUDGET, (Sx, Sy, n)
