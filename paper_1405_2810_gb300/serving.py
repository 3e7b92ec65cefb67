"""Continuous batching of LRBMS simulations over the C ABI.

Requests (a problem, its offline data and a number of online steps) arrive
at any tick. A request is admitted as soon as the context's HBM budget and
slots allow (lrbms_offline_load succeeds; LRBMS_E_BUDGET leaves it queued, in
arrival order), every tick advances all admitted simulations by one online
step in a single lrbms_step call (Algorithm 3, step 5, batched), and a
simulation that has taken its steps is read out and released, which frees
its memory for the queue. All arithmetic runs in the library's kernels; this
module only schedules. Because the kernels reduce in a fixed order per
simulation, each result is the same as the simulation run alone.

With the mixed solver a simulation recomputes its FP32 factor every
refactor_period steps, counted from its first step, and a launch lasts as
long as its slowest simulation: the factor of the largest systems is several
times their solve. Simulations that started on different ticks would put
some factor into every tick. Server(align=refactor_period) therefore starts
new simulations only on ticks that are refactor ticks of the residents, so
that all of them factor together; a request waits at most align - 1 ticks
more. It is admitted (loaded or cloned) as soon as it fits, and waits,
resident, for its start tick: the admissions of a cohort are spread over
the ticks before it starts instead of all landing in one tick.
"""
from __future__ import annotations

import time
from collections import deque
from dataclasses import dataclass, field


@dataclass
class Request:
    rid: int
    problem: dict
    offline: dict
    n_steps: int
    arrival_tick: int = 0
    sim_id: int = -1
    steps_done: int = 0
    admitted_tick: int = -1
    start_tick: int = -1     # tick of its first step
    finished_tick: int = -1
    arrival_s: float = 0.0   # wall-clock times (run_timed), seconds from its start
    admitted_s: float = -1.0
    started_s: float = -1.0  # when it joined the stepped list (its first step is the next tick)
    finished_s: float = -1.0
    admit_ms: float = 0.0    # host time of the admitting call
    result: dict = field(default_factory=dict)


class Server:
    """Admission by budget, one batched step per tick, retirement.

    backend: the ctypes binding (paper_1405_2810_gb300.lrbms) or an object
    with the same functions (lrbms_offline_load, lrbms_step, lrbms_get_state,
    lrbms_release, LrbmsError, LRBMS_E_BUDGET). admit: optional callable
    (ctx, request) -> sim_id replacing lrbms_offline_load (for instance a
    lrbms_clone of a resident simulation); it raises LrbmsError with
    LRBMS_E_BUDGET when the request does not fit yet. align: admitted
    requests start (take their first step) only on ticks t with
    (t - t0) % align == 0, t0 the first tick of the residents present since
    the server was last empty (1: on the tick after their admission)."""

    def __init__(self, backend, ctx, admit=None, align: int = 1):
        if int(align) < 1:
            raise ValueError("align must be >= 1")
        self.L = backend
        self.ctx = ctx
        self.admit = admit
        self.align = int(align)
        self.anchor = 0  # first tick of the current residents
        self.clock = None  # run_timed: seconds since its start
        self.queue: deque[Request] = deque()
        self.active: list[Request] = []
        self.ready: list[Request] = []  # admitted, waiting for their start tick
        self.done: list[Request] = []
        self.tick_ms: list[float] = []
        self.tick_n: list[int] = []  # simulations stepped per tick
        self.tick = 0
        self._next = 0

    def submit(self, problem: dict, offline: dict, n_steps: int) -> int:
        r = Request(self._next, problem, offline, int(n_steps), arrival_tick=self.tick)
        self._next += 1
        self.queue.append(r)
        return r.rid

    def _admit(self):
        if not self.active:
            self.anchor = self.tick + 1  # no residents: the next tick starts a new phase
        starting = (self.tick + 1 - self.anchor) % self.align == 0
        self._load_queued()
        if starting:  # the admitted requests take their first step in the next tick
            for r in self.ready:
                r.start_tick = self.tick + 1
                if self.clock is not None:
                    r.started_s = self.clock()
            self.active.extend(self.ready)
            self.ready = []

    def _load_queued(self):
        while self.queue:
            r = self.queue[0]
            t0 = time.perf_counter()
            try:
                if self.admit is not None:
                    r.sim_id = self.admit(self.ctx, r)
                else:
                    r.sim_id = self.L.lrbms_offline_load(self.ctx, r.problem, r.offline)
            except self.L.LrbmsError as e:
                if e.code == self.L.LRBMS_E_BUDGET:
                    break  # wait for memory to be freed; keep arrival order
                raise
            r.admit_ms = 1e3 * (time.perf_counter() - t0)
            r.admitted_tick = self.tick
            if self.clock is not None:
                r.admitted_s = self.clock()
            self.queue.popleft()
            self.ready.append(r)

    def step(self):
        """One tick: enqueue one step of every active simulation, admit the
        queued requests while it runs on the device (their copies and set-up
        kernels go to the library's admission stream), then wait for the
        step's statuses (one copy for the batch) and retire the finished
        simulations. Admitted requests join at the next start tick (with
        align 1, the next tick)."""
        ids = [r.sim_id for r in self.active]
        t0 = time.perf_counter()
        if ids:
            self.L.lrbms_step(self.ctx, ids, 1, wait=False)
        self._admit()
        if ids:
            st = self.L.lrbms_step_status(self.ctx, len(ids))
            self.tick_ms.append(1e3 * (time.perf_counter() - t0))
            self.tick_n.append(len(ids))
            still = []
            for r, code in zip(self.active[:len(ids)], st):
                r.steps_done += 1
                if code != 0 or r.steps_done >= r.n_steps:
                    r.result = self._read(r, int(code))
                    self.L.lrbms_release(self.ctx, r.sim_id)
                    r.finished_tick = self.tick
                    if self.clock is not None:
                        r.finished_s = self.clock()
                    self.done.append(r)
                else:
                    still.append(r)
            self.active = still + self.active[len(ids):]  # admitted during this tick
        self.tick += 1

    def _read(self, r: Request, code: int) -> dict:
        import numpy as np
        s = np.empty(int(r.problem["nx"]) * int(r.problem["ny"]))
        t, out = self.L.lrbms_get_state(self.ctx, r.sim_id, s)
        return {"status": code, "s": s, "t": t, "outflow": out, "steps": r.steps_done}

    def run(self, arrivals=(), max_ticks: int = 100000):
        """arrivals: iterable of (tick, problem, offline, n_steps); runs until
        every request has finished."""
        pending = sorted(arrivals, key=lambda a: a[0])
        i = 0
        while (i < len(pending) or self.queue or self.active or self.ready) and self.tick < max_ticks:
            while i < len(pending) and pending[i][0] <= self.tick:
                _, p, o, n = pending[i]
                self.submit(p, o, n)
                i += 1
            self.step()
        return sorted(self.done, key=lambda r: r.rid)

    def run_timed(self, arrivals=(), max_seconds: float = 600.0):
        """arrivals: iterable of (seconds, problem, offline, n_steps) on the wall
        clock from the call; a request is submitted once its time has come, and
        the loop sleeps only while nothing is queued or active. Runs until every
        request has finished (or max_seconds)."""
        pending = sorted(arrivals, key=lambda a: a[0])
        t0 = time.perf_counter()
        self.clock = lambda: time.perf_counter() - t0
        i = 0
        while i < len(pending) or self.queue or self.active or self.ready:
            now = self.clock()
            if now > max_seconds:
                break
            while i < len(pending) and pending[i][0] <= now:
                at, p, o, n = pending[i]
                self.submit(p, o, n)
                self.queue[-1].arrival_s = at
                i += 1
            if not self.queue and not self.active and not self.ready:
                time.sleep(max(0.0, pending[i][0] - now))
                continue
            self.step()
        self.clock = None
        return sorted(self.done, key=lambda r: r.rid)

    def latency_ms(self):
        """p50 and p99 of the per-tick step latency (host-measured, ms)."""
        import numpy as np
        if not self.tick_ms:
            return None, None
        a = np.sort(np.array(self.tick_ms))
        return float(np.percentile(a, 50)), float(np.percentile(a, 99))
