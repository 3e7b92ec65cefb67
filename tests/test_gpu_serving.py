"""Continuous batching on the GPU: simulations of different grids and basis
sizes arrive at different ticks under an HBM budget that cannot hold them all;
each one's final state equals the same simulation run alone (bitwise)."""
import numpy as np
import pytest

from lrbms_cases import abi_offline, abi_problem, case

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1405_2810_gb300 import build, lrbms
    build.build()
    return lrbms


@pytest.mark.parametrize("solver", [0, 1], ids=["fp64-solve", "mixed-solve"])
def test_staggered_arrivals_match_alone(L, solver):
    from paper_1405_2810_gb300.serving import Server
    specs = [(0, dict(name="small"), 9), (0, dict(name="rect", kind="snapshots", n=(72, 40), S=(6, 4)), 5),
             (2, dict(name="paper_bc", p_inflow=0.0), 7), (3, dict(name="small", kind="snapshots"), 4),
             (6, dict(name="strip", kind="snapshots", n=64, S=4), 6)]
    arrivals = []
    for tick, kw, n in specs:
        prob, m, co, off = case(**kw)
        arrivals.append((tick, abi_problem(prob, m), abi_offline(co, off, False), n))
    sizes = []  # resident bytes of each simulation
    for _, prob_d, off_d, _ in arrivals:
        ctx = L.lrbms_create(hbm_budget=256 << 20, max_slots=2, solver=solver)
        L.lrbms_offline_load(ctx, prob_d, off_d)
        sizes.append(L.lrbms_memory(ctx)[0])
        L.lrbms_destroy(ctx)
    # the first three arrivals cannot all be resident: the third waits for a retirement
    ctx = L.lrbms_create(hbm_budget=sum(sizes[:3]) - 4096, max_slots=8, solver=solver)
    srv = Server(L, ctx)
    done = srv.run(arrivals)
    L.lrbms_destroy(ctx)
    assert len(done) == len(specs) and all(r.result["status"] == 0 for r in done)
    assert any(r.admitted_tick > r.arrival_tick for r in done)  # the budget made someone wait
    for (tick, kw, n), r in zip(specs, done):
        ctx = L.lrbms_create(hbm_budget=64 << 20, max_slots=2, solver=solver)
        prob, m, co, off = case(**kw)
        sid = L.lrbms_offline_load(ctx, abi_problem(prob, m), abi_offline(co, off, False))
        assert L.lrbms_step(ctx, [sid], n)[0] == 0
        s = np.empty(prob.n_cells)
        t, out = L.lrbms_get_state(ctx, sid, s)
        L.lrbms_destroy(ctx)
        assert np.array_equal(s, r.result["s"]) and t == r.result["t"] and out == r.result["outflow"]
