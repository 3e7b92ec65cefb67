#!/usr/bin/env python3
"""Benchmark: batched LRBMS online steps/s and step latency on one GB300.

Workload (default, "batch"): n_sims concurrent 2D two-phase simulations on a
128x128 fine grid with 8x8 subdomains, seeded log-normal permeability
(sigma 1, correlation 0.1), viscosity ratio U[2,20] per physical dataset,
Corey relative permeabilities, M = 8 mobility profiles, requested local basis
sizes U{5..30} per subdomain (capped at the number of independent snapshot
restrictions). Offline data are built on the GPU by lrbms_offline_build from
n_prob physical datasets; every other simulation is a copy with randomly
rotated local bases (distinct bytes, identical physics). One step = one
online step (Algorithm 3, step 5) of every simulation.

Prints one JSON line. `value` is sim-steps/s with all data resident in HBM;
`e2e` is the same metric through lrbms_step_io with the saturation read from
and written to pinned host memory every step.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Batched LRBMS online steps/s and p99 step latency vs plain FP64 GPU path"
FP64_PEAK_TFLOPS = 1.26  # 152 SMs x 4 FP64 flop/clk x 2.07 GHz (measured FMA loop: 1.19)
FP32_PEAK_TFLOPS = 80.5  # 152 SMs x 128 FP32 lanes x 2 flop/clk x 2.07 GHz


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=0, help="timed steps (0: about 3 s of work)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n-sims", type=int, default=512)
    ap.add_argument("--n-prob", type=int, default=8)
    ap.add_argument("--n", type=int, default=128)
    ap.add_argument("--S", type=int, default=8)
    ap.add_argument("--n-snap", type=int, default=40)
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"],
                    help="storage of bases and components (mixed: FP32)")
    ap.add_argument("--solver", default="mixed", choices=["fp64", "mixed"],
                    help="reduced solve: FP64 Cholesky, or FP32 Cholesky with FP64 refinement")
    ap.add_argument("--refactor-period", type=int, default=0,
                    help="mixed solver: steps one FP32 factor serves (0: the library default)")
    ap.add_argument("--refactor-stages", type=int, default=1,
                    help="mixed solver: steps over which each next FP32 factor is built (default 1: in one step)")
    ap.add_argument("--horizon", type=int, default=300, help="steps per simulation (warm-up + timed)")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--cpu-workers", type=int, default=0,
                    help="oracle processes of the CPU baseline (0: host cores - 2, at most 16)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=0)
    ap.add_argument("--kernels-only", action="store_true",
                    help="profiling runs: build, warm up, run the timed steps and stop (no phase, end-to-end, "
                         "plain-path or CPU legs; the JSON line then holds only the timed value)")
    ap.add_argument("--serving", action="store_true",
                    help="continuous-batching serving run with Poisson arrivals (its own JSON line)")
    ap.add_argument("--c2", action="store_true",
                    help="C2: one simulation on the 256x256 anisotropic field (16x16 subdomains, contrast 1e6), "
                         "plain FP64 reduced steps against full fine SWIP-DG steps (its own JSON line)")
    ap.add_argument("--c2-fine-steps", type=int, default=2)
    ap.add_argument("--serve-rate", type=float, default=200.0, help="arrivals per second")
    ap.add_argument("--serve-requests", type=int, default=400)
    ap.add_argument("--serve-steps", type=int, default=300, help="online steps per request")
    ap.add_argument("--serve-align", type=int, default=0,
                    help="admit only every this many ticks (0: the refactor period, 8, with the mixed solver; "
                         "1 with FP64)")
    return ap.parse_args()


# ------------------------------------------------------------------ workload
def workload_name(a) -> str:
    return (f"{a.n_sims} concurrent 2D two-phase LRBMS simulations, {a.n}x{a.n} fine grid, "
            f"{a.S}x{a.S} subdomains, basis sizes U{{5..30}}, M=8, viscosity ratio U[2,20]")


def problem_inputs(a, p: int, rank: int = 0):
    """Seeded inputs of physical dataset p (no method arithmetic)."""
    import numpy as np
    from synth import make_problem, simplex_params, basis_sizes
    prob = make_problem("batch", sim_index=p + 1000 * rank, n=a.n, S=a.S)
    n_sub = prob.Sx * prob.Sy
    N_E = basis_sizes(n_sub, 5, 30, 31 + p + 1000 * rank)
    mu = simplex_params(a.n_snap, prob.M, 57 + p + 1000 * rank)
    return prob, N_E, mu, None


def abi_problem(prob):
    return dict(nx=prob.nx, ny=prob.ny, Sx=prob.Sx, Sy=prob.Sy, Lx=prob.Lx, Ly=prob.Ly, perm=prob.perm,
                poro=prob.poro, eta_w=prob.eta_w, eta_o=prob.eta_o,
                relperm=0 if prob.relperm == "corey" else 1, bc_type=prob.bc_type, p_D=prob.p_D,
                v_N=prob.v_N, s_D=prob.s_D, s0=prob.s0, cfl=prob.cfl, dt_mode=0, dt_fixed=0.0,
                dt_max=0.0, mean_weights=0)


def penalty_scale(prob) -> float:
    # c_pen = c_f / max(eta) with c_f = 20 max(eta)/min(eta) (penalty of Remark 1)
    return 20.0 / min(prob.eta_w, prob.eta_o)


# ------------------------------------------------------------------ CPU oracle baseline
def cpu_baseline_worker(args_dict, q, worker: int = 0):
    """Time the CPU oracle's online step (as it stands) on one simulation of
    the same workload (physical dataset worker mod n_prob), single-threaded,
    for about cpu_seconds of work."""
    try:
        for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
            os.environ[k] = "1"
        import numpy as np
        from types import SimpleNamespace
        a = SimpleNamespace(**args_dict)
        try:
            from threadpoolctl import threadpool_limits
            threadpool_limits(1)
        except Exception:
            pass
        from oracle.grid import Coarse
        from oracle.impes import FineModel
        from oracle.offline import build_offline
        from oracle.reduced import online_step
        prob, N_E, mu, _ = problem_inputs(a, worker % a.n_prob)
        m = FineModel.from_problem(prob, c_pen=penalty_scale(prob))
        co = Coarse(m.grid, prob.Sx, prob.Sy)
        t0 = time.perf_counter()
        off = build_offline(m, co, prob.s0, prob.n_steps, prob.M, kind="snapshots", mus=mu, N_E=N_E)
        t_off = time.perf_counter() - t0
        s = prob.s0.copy()
        online_step(m, off, s)  # warm-up
        n = 0
        t0 = time.perf_counter()
        while True:
            s = online_step(m, off, s)["s"]
            n += 1
            if time.perf_counter() - t0 >= a.cpu_seconds:
                break
        q.put(dict(n=n, seconds=time.perf_counter() - t0, N=int(off.N), t_off=t_off, worker=worker))
    except Exception as e:  # report, do not hide
        q.put(dict(error=repr(e), worker=worker))


def cpu_workers(a) -> int:
    return a.cpu_workers if a.cpu_workers > 0 else max(1, min(16, (os.cpu_count() or 1) - 2))


def start_cpu_baseline(a):
    """One spawned single-threaded oracle process per worker, each stepping
    its own simulation (processes, not threads: NumPy's small operations do
    not scale with BLAS threads)."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=cpu_baseline_worker, args=(vars(a), q, w), daemon=True)
             for w in range(cpu_workers(a))]
    for p in procs:
        p.start()
    return procs, q


def collect_cpu_baseline(cpu, timeout: float = 900.0) -> dict:
    """Whole-host oracle throughput: the sum over the workers of their online
    steps per second."""
    procs, q = cpu
    res = []
    t_end = time.time() + timeout
    while len(res) < len(procs) and time.time() < t_end:
        try:
            res.append(q.get(timeout=max(1.0, t_end - time.time())))
        except Exception:
            break
    for p in procs:
        p.join(timeout=5)
    bad = [r for r in res if "error" in r]
    if bad or len(res) < len(procs):
        return {"error": bad[0]["error"] if bad else f"{len(procs) - len(res)} oracle workers did not finish"}
    value = sum(r["n"] / r["seconds"] for r in res)
    n = sum(r["n"] for r in res)
    return dict(value=value, unit="sim-steps/s", cores=len(res), kind="oracle",
                sample=f"{len(res)} single-threaded processes, one simulation each of the same workload "
                       f"(N = {min(r['N'] for r in res)}..{max(r['N'] for r in res)}), {n} online steps in "
                       f"about {res[0]['seconds']:.0f} s each, NumPy/SciPy FP64; offline builds "
                       f"(about {max(r['t_off'] for r in res):.0f} s) not timed")


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.rows = []
        self.proc = None
        self.th = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.th = threading.Thread(target=self._read, daemon=True)
        self.th.start()

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        if self.th:
            self.th.join(timeout=2)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[0]))
                mx = float(r[1])
            except (ValueError, IndexError):
                continue
            for k, nm in enumerate(names):
                if len(r) > 4 + k and r[4 + k].lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ algorithmic work
def solve_flops(N_E, Sx: int) -> tuple:
    """Flops of the reduced solve per simulation, as implemented: the envelope
    block Cholesky (with the products by the diagonal inverses), one forward
    and backward substitution pair, and one FP64 block mat-vec A x."""
    n = len(N_E)
    xoff = [0]
    for v in N_E:
        xoff.append(xoff[-1] + int(v))
    fl = 0.0
    for k in range(n):
        jl = max(0, k - Sx)
        Nk = N_E[k]
        for j in range(jl, k + 1):
            Nj = N_E[j]
            ln = xoff[j] - xoff[jl]
            if j < k:
                fl += 2.0 * Nk * Nj * ln + Nk * Nj * (Nj + 1)
            else:
                fl += Nk * (Nk + 1) * ln + 2.0 * Nk ** 3 / 3.0
    subst = 0.0
    for k in range(n):
        jl = max(0, k - Sx)
        W = xoff[k + 1] - xoff[jl]
        subst += 2.0 * 2.0 * N_E[k] * (W - N_E[k]) + 2.0 * N_E[k] * (N_E[k] + 1)
    nnz = sum(int(v) ** 2 for v in N_E)
    for e in range(n):
        if e % Sx < Sx - 1 and e + 1 < n:
            nnz += 2 * N_E[e] * N_E[e + 1]
        if e + Sx < n:
            nnz += 2 * N_E[e] * N_E[e + Sx]
    return fl, subst, 2.0 * nnz


def stream_bytes(N_E, Sx: int, cells: int, M: int, elem: int) -> dict:
    """Algorithmic bytes per simulation of the streaming phases."""
    n = len(N_E)
    a = sum(int(v) ** 2 for v in N_E)
    for e in range(n):
        if e % Sx < Sx - 1 and e + 1 < n:
            a += N_E[e] * N_E[e + 1]
        if e + Sx < n:
            a += N_E[e] * N_E[e + Sx]
    N = int(sum(N_E))
    return {"assemble": (M + 1) * a * elem + a * 8 + (M + 1) * N * 8 + N * 8,
            "reconstruct": sum(3 * cells * int(v) * elem for v in N_E) + 24 * cells * n + 8 * N}


def solve_info(L, ctx, ids):
    """Per-simulation reduced-solve counters (LRBMS_FIELD_SOLVE_INFO)."""
    import numpy as np
    return np.array([L.lrbms_get_field(ctx, i, L.FIELD_SOLVE_INFO, dtype=np.int32) for i in ids], dtype=np.int64)


# ------------------------------------------------------------------ multi-rank aggregation
def max_over_ranks(x: float, dist=None, device: str = "cpu") -> float:
    """Largest value of x over all ranks (x itself without a process group)."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(n_sims: int, steps: int, seconds: float, world: int) -> float:
    """Whole-job sim-steps/s: each of `world` ranks advances its own n_sims
    simulations `steps` times (weak scaling, no data-path collective)."""
    return world * n_sims * steps / seconds


# ------------------------------------------------------------------ main arms
def run_reference(a, rank: int, world: int):
    if rank != 0:
        return
    r = collect_cpu_baseline(start_cpu_baseline(a))
    if "error" in r:
        print(json.dumps({"impl": "reference", "unavailable": f"oracle baseline failed: {r['error']}"}))
        return
    line = {"impl": "reference", "metric": METRIC, "value": r["value"], "unit": r["unit"], "n_gpus": world,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1000.0 / r["value"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(a), "sample": r["sample"]},
            "cpu_baseline": {"value": r["value"], "unit": r["unit"], "cores": r["cores"], "kind": "oracle",
                             "sample": r["sample"]},
            "e2e": {"value": r["value"], "unit": r["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


SERVE_SHAPES = ((64, 4), (64, 8), (64, 16), (128, 8), (128, 16))  # (grid n, subdomains S), n / S >= 4


def run_serving(a):
    """Continuous batching under Poisson arrivals: every request is a
    simulation of one of SERVE_SHAPES (a seeded physical dataset per shape,
    built offline on the GPU and kept resident as a pool) admitted as a copy
    of its pool entry, advanced one online step per tick with every other
    active simulation, and released after serve_steps steps. Reports the
    per-tick step latency (p50/p99), the admission time apart from it, the
    request latency (arrival to finish) and the sustained throughput."""
    import numpy as np
    import torch
    from types import SimpleNamespace
    from paper_1405_2810_gb300 import build, lrbms as L
    from paper_1405_2810_gb300.serving import Server
    build.build()
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    free, _tot = torch.cuda.mem_get_info()
    prec = L.LRBMS_FP64 if a.precision == "fp64" else L.LRBMS_MIXED
    solver = L.LRBMS_SOLVE_MIXED if a.solver == "mixed" else L.LRBMS_SOLVE_FP64
    period = a.refactor_period if a.refactor_period > 0 else 8  # FP32 refactor period of the mixed solver
    stages = max(a.refactor_stages, 1)
    ctx = L.lrbms_create(precision=prec, max_slots=2048, hbm_budget=int(min(free * 0.45, 96 << 30)),
                         stream=stream.cuda_stream, solver=solver, refactor_period=period,
                         refactor_stages=stages if a.solver == "mixed" else 0)
    t0 = time.perf_counter()
    pool = []  # (sim id, nx, ny, shape)
    for i, (n, S) in enumerate(SERVE_SHAPES):
        prob, N_E, mu, _ = problem_inputs(SimpleNamespace(n=n, S=S, n_snap=a.n_snap), 500 + i)
        (sid,) = L.lrbms_offline_build(ctx, [abi_problem(prob)], [dict(M=prob.M, n_steps_T=prob.n_steps, N_E=N_E,
                                       mu=mu, c_pen=penalty_scale(prob), allow_fewer=1)], 1)
        pool.append((sid, prob.nx, prob.ny, f"{n}x{n}/{S}x{S}"))
    t_pool = time.perf_counter() - t0
    rng = np.random.default_rng(np.random.PCG64(1405))
    times = np.cumsum(rng.exponential(1.0 / a.serve_rate, size=a.serve_requests))
    kinds = rng.integers(0, len(pool), size=a.serve_requests)
    arrivals = [(float(t), {"nx": pool[k][1], "ny": pool[k][2]}, {"src": pool[k][0], "kind": int(k)},
                 a.serve_steps) for t, k in zip(times, kinds)]
    align = a.serve_align if a.serve_align > 0 else (period if a.solver == "mixed" else 1)
    srv = Server(L, ctx, admit=lambda c, r: L.lrbms_clone(c, r.offline["src"], None), align=align)
    t1 = time.perf_counter()
    done = srv.run_timed(arrivals)
    wall = time.perf_counter() - t1
    ok = sum(1 for r in done if r.result.get("status") == 0)
    p50, p99 = srv.latency_ms()
    lat = np.array([r.finished_s - r.arrival_s for r in done])
    wait = np.array([r.admitted_s - r.arrival_s for r in done])
    start_wait = np.array([r.started_s - r.arrival_s for r in done])
    adm = np.array([r.admit_ms for r in done])
    steps = sum(r.steps_done for r in done)
    print(json.dumps({
        "metric": "LRBMS serving: per-tick step latency under Poisson arrivals of mixed grids",
        "value": p99, "unit": "ms (p99 step latency)", "higher_is_better": False,
        "p50_step_ms": p50, "p99_step_ms": p99, "ticks": len(srv.tick_ms),
        "step_ms_percentiles": {str(q): float(np.percentile(srv.tick_ms, q)) for q in (90, 95, 100)},
        "throughput_sim_steps_per_s": steps / wall,
        "request_latency_s": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99))},
        "admission_wait_s": {"p50": float(np.percentile(wait, 50)), "p99": float(np.percentile(wait, 99))},
        "start_wait_s": {"p50": float(np.percentile(start_wait, 50)), "p99": float(np.percentile(start_wait, 99))},
        "admission_ms": {"p50": float(np.percentile(adm, 50)), "p99": float(np.percentile(adm, 99))},
        "active_sims": {"mean": float(np.mean(srv.tick_n)), "max": int(max(srv.tick_n))},
        "requests": len(done), "requests_ok": ok, "sim_steps": steps, "wall_s": wall,
        "dtype": "f64+f32" if a.solver == "mixed" else "f64", "data": "synthetic",
        "config": {"workload": f"Poisson arrivals at {a.serve_rate:g}/s, {a.serve_requests} requests of "
                               f"{a.serve_steps} steps, grids/subdomains " + ", ".join(p[3] for p in pool),
                   "precision": a.precision, "solver": a.solver, "admission_align_ticks": align,
                   "refactor_stages": stages if a.solver == "mixed" else None,
                   "pool_build_s": t_pool},
    }))
    L.lrbms_destroy(ctx)


def run_c2(a):
    """C2: one simulation of the 256x256 anisotropic workload (correlation
    lengths 0.2 x 0.02, contrast 1e6, viscosity ratio 5, 16x16 subdomains,
    local bases of at most 20 functions from 24 snapshots built on the GPU).
    Times plain FP64 reduced steps (FP64 block Cholesky every step, one
    simulation per call, waiting for each step) and full fine SWIP-DG steps
    (Algorithm 1 through lrbms_fine_step) from the same state."""
    import numpy as np
    import torch
    from paper_1405_2810_gb300 import build, lrbms as L
    from synth import make_problem, simplex_params
    build.build()
    prob = make_problem("aniso")
    n_sub = prob.Sx * prob.Sy
    ctx = L.lrbms_create(precision=L.LRBMS_FP64, solver=L.LRBMS_SOLVE_FP64, max_slots=4, hbm_budget=8 << 30)
    t0 = time.perf_counter()
    (sid,), sizes = L.lrbms_offline_build(ctx, [abi_problem(prob)], [dict(
        M=prob.M, n_steps_T=prob.n_steps, N_E=np.full(n_sub, 20, dtype=np.int32),
        mu=simplex_params(24, prob.M, 2811), c_pen=penalty_scale(prob), allow_fewer=1)], 1, None,
        return_sizes=True)
    t_build = time.perf_counter() - t0
    fine = L.lrbms_clone(ctx, sid, None)
    L.lrbms_step(ctx, [sid], 3)  # warm-up (also the autotuner)
    K = 20
    t0 = time.perf_counter()
    for _ in range(K):
        st = L.lrbms_step(ctx, [sid], 1)
    t_red = (time.perf_counter() - t0) / K
    s_now = L.lrbms_get_field(ctx, sid, L.FIELD_S)
    L.lrbms_set_saturation(ctx, fine, s_now)
    L.lrbms_fine_step(ctx, [fine], 1)  # warm-up (allocation, code load)
    L.lrbms_set_saturation(ctx, fine, s_now)
    t0 = time.perf_counter()
    stf = L.lrbms_fine_step(ctx, [fine], a.c2_fine_steps)
    t_fine = (time.perf_counter() - t0) / a.c2_fine_steps
    print(json.dumps({
        "metric": "C2: plain FP64 reduced step vs full fine SWIP-DG step, one simulation",
        "value": t_fine / t_red, "unit": "x (fine step time / reduced step time)", "higher_is_better": True,
        "reduced_step_ms": 1e3 * t_red, "fine_step_ms": 1e3 * t_fine, "reduced_status": int(st[0]),
        "fine_status": int(stf[0]), "basis_sizes_mean": float(sizes.mean()), "N": int(sizes.sum()),
        "offline_build_s": t_build, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "256x256 anisotropic log-normal field (0.2 x 0.02, contrast 1e6), 16x16 subdomains, "
                               "viscosity ratio 5, M=8, basis sizes <= 20",
                   "reduced": "FP64 block Cholesky every step, one refinement step",
                   "fine": "SWIP-DG P1 (3 x 65536 unknowns), FP64 envelope block Cholesky, one CTA"},
    }))
    L.lrbms_destroy(ctx)


def main():
    a = parse_args()
    if a.serving:
        run_serving(a)
        return
    if a.c2:
        run_c2(a)
        return
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if a.impl == "reference":
        run_reference(a, rank, world)
        return
    cpu = None
    if rank == 0 and world == 1 and not a.no_cpu_baseline and not a.kernels_only:
        cpu = start_cpu_baseline(a)  # spawned before the first GPU call

    import numpy as np
    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device(f"cuda:{local}"))
    from paper_1405_2810_gb300 import build, lrbms as L
    from synth import random_orthogonal
    build.build()

    stream = torch.cuda.Stream()  # a real stream: the library and the events share it
    torch.cuda.set_stream(stream)
    free, _tot = torch.cuda.mem_get_info()
    budget = int(min(free * 0.45, 96 << 30))
    prec = L.LRBMS_FP64 if a.precision == "fp64" else L.LRBMS_MIXED
    solver = L.LRBMS_SOLVE_MIXED if a.solver == "mixed" else L.LRBMS_SOLVE_FP64
    ctx = L.lrbms_create(precision=prec, max_slots=a.n_sims + 8, hbm_budget=budget,
                         stream=stream.cuda_stream, device=local, solver=solver,
                         refactor_period=a.refactor_period, refactor_stages=max(a.refactor_stages, 1))

    # ---- offline data on the GPU (not timed)
    t0 = time.perf_counter()
    n_copies = a.n_sims // a.n_prob
    assert n_copies * a.n_prob == a.n_sims, "n_sims must be a multiple of n_prob"
    ids, sizes = [], []
    rng = np.random.default_rng(2024 + rank)
    per_call = 4
    for p0 in range(0, a.n_prob, per_call):
        probs, opts, rots = [], [], []
        for p in range(p0, min(a.n_prob, p0 + per_call)):
            prob, N_E, mu, _ = problem_inputs(a, p, rank)
            probs.append(abi_problem(prob))
            opts.append(dict(M=prob.M, n_steps_T=prob.n_steps, N_E=N_E, mu=mu, c_pen=penalty_scale(prob),
                             allow_fewer=1))
            rots.append(N_E)
        got_ids, got = L.lrbms_offline_build(ctx, probs, opts, 1, None, return_sizes=True)
        for k, sid in enumerate(got_ids):
            ids.append(sid)
            sizes.append(got[k])
            for r in range(1, n_copies):  # copies with randomly rotated local bases
                Q = np.concatenate([random_orthogonal(int(v), rng).reshape(-1) for v in got[k]])
                ids.append(L.lrbms_clone(ctx, sid, Q))
    t_build = time.perf_counter() - t0
    sizes = np.array(sizes)
    N_mean = float(sizes.sum(axis=1).mean())
    used, cap = L.lrbms_memory(ctx)

    # ---- warm-up
    st = L.lrbms_step(ctx, ids, max(a.warmup, 1))
    assert np.all(st == 0), f"warm-up status {np.unique(st)}"
    # steps for about 3 s if not given
    K = a.steps
    if K <= 0:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        L.lrbms_step(ctx, ids, 1, wait=False)
        e1.record(stream)
        torch.cuda.synchronize()
        K = max(10, int(math.ceil(3000.0 / max(e0.elapsed_time(e1), 1e-3))))
        K = min(K, a.horizon - max(a.warmup, 1) - 40)  # stay within the simulated horizon

    # ---- timed region: device-resident inputs
    info0 = solve_info(L, ctx, ids)
    clocks = ClockSampler(local)
    clocks.start()
    launches0 = L.lrbms_launch_count(ctx)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    # one lrbms_step call per step (one graph launch each), an event between
    # consecutive steps for the per-step latency
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(K + 1)]
    evs[0].record(stream)
    for k in range(K):
        L.lrbms_step(ctx, ids, 1, wait=False)
        evs[k + 1].record(stream)
    torch.cuda.synchronize()
    elapsed_ms = evs[0].elapsed_time(evs[K])
    step_lat_ms = [evs[k].elapsed_time(evs[k + 1]) for k in range(K)]
    launches = L.lrbms_launch_count(ctx) - launches0
    clk = clocks.stop()
    elapsed_ms = max_over_ranks(elapsed_ms, dist, "cuda")
    status = L.lrbms_step(ctx, ids, 0)
    n_ok = int(np.sum(status == 0))
    value = job_throughput(a.n_sims, K, elapsed_ms / 1000.0, world)
    # reduced-solve work of the timed steps (per simulation: substitution
    # passes, FP32 factorisations, FP64 redos)
    dinfo = solve_info(L, ctx, ids) - info0
    solves = np.maximum(dinfo[:, 5], 1)
    passes_per_solve = dinfo[:, 4] / solves
    factor_rate = dinfo[:, 2] / solves

    # ---- per-phase and per-step times: Kp further steps launched kernel by
    # kernel with CUDA events between the phases (not part of `value`)
    Kp = max(3, min(10, K))
    L.lrbms_profile_start(ctx, Kp)
    L.lrbms_step(ctx, ids, Kp, wait=False)
    phase_ms, _ = L.lrbms_profile_read(ctx, Kp)

    if a.kernels_only:
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": value, "unit": "sim-steps/s", "steps": K,
                              "ms_per_step": elapsed_ms / K, "sims_ok": n_ok, "kernels_only": True}))
        L.lrbms_destroy(ctx)
        if dist:
            dist.destroy_process_group()
        return

    # ---- end to end through lrbms_step_io with pinned host buffers
    n_cells = a.n * a.n
    Ke = a.e2e_steps or max(3, min(K, 20))
    s_in = [torch.zeros(n_cells, dtype=torch.float64).pin_memory() for _ in ids]
    s_out = [torch.empty(n_cells, dtype=torch.float64).pin_memory() for _ in ids]
    L.lrbms_step_io(ctx, ids, 1, None, s_out)  # current state -> host
    for i in range(len(ids)):
        s_in[i].copy_(s_out[i])
    L.lrbms_step_io(ctx, ids, 1, s_in, s_out)  # warm-up of the io path
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(Ke):
        for i in range(len(ids)):
            s_in[i], s_out[i] = s_out[i], s_in[i]
        L.lrbms_step_io(ctx, ids, 1, s_in, s_out)
    e2e_s = max_over_ranks(time.perf_counter() - t0, dist, "cuda")
    e2e_value = job_throughput(a.n_sims, Ke, e2e_s, world)

    # ---- plain FP64 single-simulation path: one simulation, one step per call
    ctx1 = L.lrbms_create(precision=L.LRBMS_FP64, max_slots=2, hbm_budget=1 << 30, device=local)
    prob, N_E, mu, _ = problem_inputs(a, 0, rank)
    (one,) = L.lrbms_offline_build(ctx1, [abi_problem(prob)], [dict(M=prob.M, n_steps_T=prob.n_steps,
                                   N_E=sizes[0], mu=mu, c_pen=penalty_scale(prob))], 1)
    L.lrbms_step(ctx1, [one], 3)
    n1 = max(5, min(50, K))
    t0 = time.perf_counter()
    for _ in range(n1):
        L.lrbms_step(ctx1, [one], 1)
    plain = n1 / (time.perf_counter() - t0)
    L.lrbms_destroy(ctx1)

    fp64_redos = int(dinfo[:, 1].sum())
    stale_retries = int(dinfo[:, 3].sum())

    # ---- roofline of the dominant phase
    names = L.PHASES
    dom = int(np.argmax(phase_ms))
    Sx = a.S
    cells = (a.n // a.S) ** 2
    elem = 8 if a.precision == "fp64" else 4
    if names[dom] == "solve":
        # per simulation and step: FP32 factorisations x factor flops, substitution
        # passes x (forward + backward) flops in the factor's type; mixed (conjugate
        # gradients): the initial residual and one FP64 block mat-vec per pass, plus
        # the pass's two dot products and three vector updates (10 N); FP64: one
        # residual per refinement
        f_lo = f_hi = 0.0
        for k, sz in enumerate(sizes):
            fac, sub, res = solve_flops(list(sz), Sx)
            sl = slice(k * n_copies, (k + 1) * n_copies)  # ids are grouped by physical dataset
            if a.solver == "mixed":
                f_lo += float(np.sum(factor_rate[sl] * fac + passes_per_solve[sl] * sub))
                f_hi += float(np.sum((passes_per_solve[sl] + 1) * res + passes_per_solve[sl] * 10.0 * float(sum(sz))))
            else:
                f_hi += float(np.sum(fac + passes_per_solve[sl] * sub + (passes_per_solve[sl] - 1) * res))
        t_solve = phase_ms[dom] / 1000.0
        t_min = f_lo / (FP32_PEAK_TFLOPS * 1e12) + f_hi / (FP64_PEAK_TFLOPS * 1e12)
        work = (f_lo + f_hi) * 1e-12
        roof = {"bound": "alu",
                "kernel": "k_factor32 + k_refine32 + k_retry32" if a.solver == "mixed" else "k_csolve64",
                "achieved": work / t_solve, "peak": work / t_min, "unit": "TFLOP/s", "frac": t_min / t_solve,
                "traffic": None,
                "peak_source": ("time-weighted ALU peak of the solve's FP32 and FP64 flops: "
                                "FP32 152 SMs x 256 flop/clk, FP64 152 SMs x 4 flop/clk, at 2.07 GHz "
                                "(recipe unit counts and clock)"),
                "flops_fp32": f_lo, "flops_fp64": f_hi}
    else:
        sb = [stream_bytes(list(sz), Sx, cells, 8, elem) for sz in sizes]
        key = names[dom] if names[dom] in sb[0] else None
        byt = sum(b.get(key, 0) for b in sb) * n_copies if key else 0
        achieved = byt / (phase_ms[dom] / 1000.0) / 1e9
        peak = float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"]) \
            if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else 6800.0
        roof = {"bound": "hbm", "kernel": names[dom], "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": None}

    cpu_line = None
    if cpu is not None:
        r = collect_cpu_baseline(cpu)
        cpu_line = r if "error" in r else {k: r[k] for k in ("value", "unit", "cores", "kind", "sample")}

    if rank == 0:
        steps_sorted = sorted(step_lat_ms)
        p50 = steps_sorted[len(steps_sorted) // 2]
        p99 = steps_sorted[min(len(steps_sorted) - 1, int(math.ceil(0.99 * len(steps_sorted))) - 1)]
        line = {
            "metric": METRIC, "value": value, "unit": "sim-steps/s", "n_gpus": world, "steps": K,
            "warmup": a.warmup, "ms_per_step": elapsed_ms / K, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None,
            "dtype": ("f64" if a.solver == "fp64" else "f64+f32") if a.precision == "fp64" else "f32+f64",
            "data": "synthetic",
            "config": {"workload": workload_name(a), "n_sims": a.n_sims, "physical_datasets": a.n_prob,
                       "grid": f"{a.n}x{a.n}", "subdomains": f"{a.S}x{a.S}", "M": 8,
                       "basis_sizes_mean_N": N_mean, "precision": a.precision, "solver": a.solver,
                       "refactor_stages": max(a.refactor_stages, 1),
                       "l2": f"inputs larger than L2: {used / 2**30:.1f} GiB resident",
                       "p50_step_ms": p50, "p99_step_ms": p99, "sims_ok": n_ok,
                       "offline_build_s": t_build, "parallelism": f"replicas x{world}",
                       "passes_per_solve": float(passes_per_solve.mean()),
                       "fp32_factorisations_per_step": float(factor_rate.mean()),
                       "stale_factor_retries": stale_retries, "fp64_redos": fp64_redos},
            "phases_ms": {n: float(v) for n, v in zip(names, phase_ms)},
            "roofline": roof,
            "plain_fp64_single_sim_steps_per_s": plain,
            "vs_plain_fp64_single_sim": value / plain,
            "e2e": {"value": e2e_value, "unit": "sim-steps/s", "h2d_bytes_per_step": 8 * n_cells * a.n_sims,
                    "d2h_bytes_per_step": 8 * n_cells * a.n_sims},
            "gpu_launches": int(launches),
            "clocks": clk,
            "cpu_baseline": cpu_line,
        }
        print(json.dumps(line))
    L.lrbms_destroy(ctx)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
