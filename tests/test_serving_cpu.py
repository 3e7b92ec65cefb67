"""Serving loop logic (admission by budget in arrival order, one batched step
per tick, retirement) against a fake backend on CPU."""
import numpy as np
import pytest

from paper_1405_2810_gb300.serving import Server


class FakeLib:
    LRBMS_E_BUDGET = -2

    class LrbmsError(Exception):
        def __init__(self, code, msg=""):
            super().__init__(msg)
            self.code = code

    def __init__(self, capacity):
        self.capacity = capacity  # simultaneous simulations
        self.live = {}
        self.next_id = 0
        self.calls = []

    def lrbms_offline_load(self, ctx, problem, offline):
        if len(self.live) >= self.capacity:
            raise self.LrbmsError(self.LRBMS_E_BUDGET, "budget")
        sid = self.next_id
        self.next_id += 1
        self.live[sid] = {"steps": 0, "nx": problem["nx"], "ny": problem["ny"]}
        return sid

    def lrbms_step(self, ctx, ids, n, wait=True):
        self.calls.append(list(ids))
        for i in ids:
            self.live[i]["steps"] += n
        self.pending = np.zeros(len(ids), dtype=np.int32)
        return self.pending if wait else None

    def lrbms_step_status(self, ctx, n):
        return self.pending[:n]

    def lrbms_get_state(self, ctx, sid, s):
        s[:] = self.live[sid]["steps"]
        return float(self.live[sid]["steps"]), 0.0

    def lrbms_release(self, ctx, sid):
        del self.live[sid]


def test_admission_in_arrival_order_and_retirement():
    lib = FakeLib(capacity=2)
    srv = Server(lib, ctx=None)
    prob = {"nx": 2, "ny": 2}
    arrivals = [(0, prob, None, 3), (0, prob, None, 1), (0, prob, None, 2), (4, prob, None, 2)]
    done = srv.run(arrivals)
    assert [r.rid for r in done] == [0, 1, 2, 3]
    assert all(r.result["steps"] == r.n_steps for r in done)
    assert all(np.all(r.result["s"] == r.n_steps) for r in done)
    # at most two simulations live at once; request 2 waits for request 1 to retire
    assert max(len(c) for c in lib.calls) == 2
    assert done[2].admitted_tick == done[1].finished_tick + 1
    assert not lib.live  # every slot released


def test_budget_error_other_than_budget_is_raised():
    class Broken(FakeLib):
        def lrbms_offline_load(self, ctx, problem, offline):
            raise self.LrbmsError(-7, "format")
    srv = Server(Broken(1), ctx=None)
    srv.submit({"nx": 1, "ny": 1}, None, 1)
    with pytest.raises(Broken.LrbmsError):
        srv.step()


def test_admit_hook_and_timed_arrivals():
    """The admission hook replaces offline loading (clones of a resident pool);
    wall-clock arrivals are submitted once due and every request finishes."""
    lib = FakeLib(capacity=3)
    made = []

    def admit(ctx, r):
        made.append(r.offline["src"])
        return lib.lrbms_offline_load(ctx, r.problem, None)

    srv = Server(lib, ctx=None, admit=admit)
    prob = {"nx": 1, "ny": 2}
    arrivals = [(0.0, prob, {"src": 7}, 2), (0.0, prob, {"src": 8}, 3), (0.02, prob, {"src": 9}, 1),
                (0.05, prob, {"src": 7}, 2), (0.05, prob, {"src": 8}, 2)]
    done = srv.run_timed(arrivals)
    assert [r.rid for r in done] == [0, 1, 2, 3, 4]
    assert made == [7, 8, 9, 7, 8]  # admitted in arrival order through the hook
    assert all(r.result["steps"] == r.n_steps for r in done)
    assert all(r.arrival_s <= r.admitted_s <= r.finished_s for r in done)
    assert done[3].arrival_s == 0.05 and done[3].admitted_s >= 0.05
    assert max(len(c) for c in lib.calls) <= 3 and not lib.live


def test_aligned_admission_keeps_residents_in_phase():
    """With align=k every simulation takes its first step on a tick that is a
    multiple of k after the first tick of the residents, so their step counts
    agree modulo k (the mixed solver's refactor ticks coincide). Requests are
    admitted (loaded) as soon as they arrive and wait, resident, for their
    start tick; an empty server starts a new phase at once."""
    lib = FakeLib(capacity=100)
    srv = Server(lib, ctx=None, align=4)
    prob = {"nx": 1, "ny": 1}
    arrivals = [(0, prob, None, 10), (1, prob, None, 10), (2, prob, None, 3), (5, prob, None, 6),
                (9, prob, None, 2), (30, prob, None, 5), (31, prob, None, 4)]
    done = srv.run(arrivals)
    assert [r.rid for r in done] == list(range(len(arrivals)))
    assert all(r.result["steps"] == r.n_steps for r in done)
    assert all(r.admitted_tick == r.arrival_tick for r in done)  # loaded on arrival
    starts = [r.start_tick for r in done]
    assert starts[0] == 1  # request 0 is admitted on tick 0, which steps nothing
    assert all((s - starts[0]) % 4 == 0 for s in starts[:5])
    assert all(0 < s - r.arrival_tick <= 4 for s, r in zip(starts, done))
    # the server emptied before request 5 arrived: it starts a new phase at once
    assert starts[5] == done[5].arrival_tick + 1
    assert (starts[6] - starts[5]) % 4 == 0
    # every step call lists only started simulations, each with its steps counted from its start
    assert all(r.finished_tick - r.start_tick + 1 == r.n_steps for r in done)
    assert not lib.live
    with pytest.raises(ValueError):
        Server(lib, ctx=None, align=0)


def test_aligned_admission_waits_for_budget_in_order():
    """A request that does not fit stays queued (arrival order kept) and is
    loaded once a retirement frees memory; it still starts on a start tick."""
    lib = FakeLib(capacity=2)
    srv = Server(lib, ctx=None, align=3)
    prob = {"nx": 1, "ny": 1}
    done = srv.run([(0, prob, None, 4), (0, prob, None, 7), (1, prob, None, 2), (2, prob, None, 2)])
    assert [r.rid for r in done] == [0, 1, 2, 3]
    assert all(r.result["steps"] == r.n_steps for r in done)
    assert max(len(c) for c in lib.calls) <= 2
    assert done[2].admitted_tick >= done[0].finished_tick  # waited for request 0's memory
    starts = [r.start_tick for r in done]
    assert all((s - starts[0]) % 3 == 0 for s in starts if s <= done[1].finished_tick)
    assert not lib.live
