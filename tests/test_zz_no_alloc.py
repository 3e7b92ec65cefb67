"""The allocation-free reduced solve (lrbms_solve_noalloc) against the solve
inside lrbms_step. The entry point exists for callers that cannot call
cudaMalloc (device memory owned by another allocator, or a time-critical loop
where an allocation's synchronisation or failure is not allowed); its working
memory is a fixed array in device memory. Two calls in a row check that
leftover contents of that shared array do not leak into the next result."""
import numpy as np
import pytest

from lrbms_cases import abi_offline, abi_problem, case, rel

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


@pytest.mark.parametrize("solver", [0, 1], ids=["fp64-solve", "mixed-solve"])
def test_noalloc_solve_matches_step_twice(L, solver):
    import torch
    prob, m, co, off = c = case("small", kind="snapshots")
    ctx = L.lrbms_create(hbm_budget=256 << 20, max_slots=2, solver=solver)
    sid = L.lrbms_offline_load(ctx, abi_problem(prob, m), abi_offline(co, off))
    for call in range(2):  # a different system on each call (the state advances)
        assert L.lrbms_step(ctx, [sid], 1)[0] == 0
        A = torch.from_numpy(L.lrbms_get_field(ctx, sid, L.FIELD_A)).cuda()
        b = torch.from_numpy(L.lrbms_get_field(ctx, sid, L.FIELD_RHS)).cuda()
        x_ref = L.lrbms_get_field(ctx, sid, L.FIELD_X)
        x = torch.full_like(b, np.nan)
        rc = L.lrbms_solve_noalloc(prob.Sx, prob.Sy, off.N_E, A, b, x, solver=solver)
        assert rc == L.LRBMS_OK
        assert rel(x.cpu().numpy(), x_ref) < TOL, call
    L.lrbms_destroy(ctx)


def test_noalloc_rejects_oversized_system(L):
    import torch
    NE = np.full(64 * 64, 32, dtype=np.int32)  # factor far beyond the fixed array
    A = torch.zeros(1, dtype=torch.float64, device="cuda")
    rc = L.lrbms_solve_noalloc(64, 64, NE, A, A, A)
    assert rc == L.LRBMS_E_BUDGET
