"""ctypes binding of the C ABI in include/lrbms.h.

Argument marshalling only: every step of the online scheme runs in the CUDA
kernels of liblrbms.so. Arrays may be NumPy arrays (host) or objects with a
``data_ptr()`` method such as CUDA torch tensors (device); they must be
C-contiguous with the dtype the header states. If the shared library is
missing, every call raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblrbms.so")

LRBMS_OK = 0
LRBMS_E_ARG = -1
LRBMS_E_BUDGET = -2
LRBMS_E_CUDA = -3
LRBMS_E_NOT_SPD = -4
LRBMS_E_NONFINITE = -5
LRBMS_E_TIMEOUT = -6
LRBMS_E_FORMAT = -7
LRBMS_E_CFL = -8
LRBMS_E_STATE = -9
LRBMS_FP64 = 0
LRBMS_MIXED = 1
LRBMS_COREY = 0
LRBMS_LINEAR = 1
LRBMS_DT_CFL = 0
LRBMS_DT_FIXED = 1
LRBMS_VELOCITY_STATE = 0
LRBMS_VELOCITY_FITTED = 1
LRBMS_TRANSPORT_FV = 0
LRBMS_TRANSPORT_DG1 = 1
LRBMS_SOLVE_FP64 = 0
LRBMS_SOLVE_MIXED = 1
FIELD_THETA, FIELD_A, FIELD_RHS, FIELD_X, FIELD_P, FIELD_FLUX, FIELD_S, FIELD_DT, FIELD_STATUS, FIELD_SOLVE_INFO, \
    FIELD_SLOPES, FIELD_PHI = range(12)

EXPORTED = ["lrbms_create", "lrbms_destroy", "lrbms_offline_load", "lrbms_offline_build",
            "lrbms_release", "lrbms_clone", "lrbms_step", "lrbms_step_io", "lrbms_profile_start", "lrbms_profile_read",
            "lrbms_run", "lrbms_get_state", "lrbms_set_saturation", "lrbms_get_field",
            "lrbms_field_bytes", "lrbms_sync", "lrbms_memory", "lrbms_launch_count", "lrbms_solve_noalloc",
            "lrbms_fine_step", "lrbms_step_status", "lrbms_test_withhold_copy", "lrbms_test_factor_plan",
            "lrbms_tuned_threads", "lrbms_last_error", "lrbms_set_slopes"]


class LrbmsError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"lrbms error {code}: {msg}")
        self.code = code


class Config(C.Structure):
    _fields_ = [("precision", C.c_int), ("max_slots", C.c_int), ("hbm_budget", C.c_size_t),
                ("stream", C.c_void_p), ("device", C.c_int), ("solver", C.c_int),
                ("refine_iters", C.c_int), ("refactor_period", C.c_int), ("refactor_stages", C.c_int)]


class Problem(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("Sx", C.c_int), ("Sy", C.c_int),
                ("Lx", C.c_double), ("Ly", C.c_double),
                ("perm", C.c_void_p), ("poro", C.c_void_p),
                ("eta_w", C.c_double), ("eta_o", C.c_double), ("relperm", C.c_int),
                ("bc_type", C.c_void_p), ("p_D", C.c_void_p), ("v_N", C.c_void_p),
                ("s_D", C.c_void_p), ("s0", C.c_void_p),
                ("cfl", C.c_double), ("dt_mode", C.c_int), ("dt_fixed", C.c_double),
                ("dt_max", C.c_double), ("mean_weights", C.c_int), ("velocity", C.c_int),
                ("transport", C.c_int)]


class Offline(C.Structure):
    _fields_ = [("M", C.c_int), ("N_E", C.c_void_p), ("prof_idx", C.c_void_p), ("prof", C.c_void_p),
                ("Gpinv", C.c_void_p), ("Phi", C.c_void_p), ("Dblk", C.c_void_p),
                ("Fblk", C.c_void_p), ("rhs", C.c_void_p), ("c_pen", C.c_double), ("Lf", C.c_double)]


class BuildOpts(C.Structure):
    _fields_ = [("M", C.c_int), ("n_steps_T", C.c_int), ("N_E", C.c_void_p), ("n_snap", C.c_int),
                ("mu", C.c_void_p), ("c_pen", C.c_double), ("allow_fewer", C.c_int), ("greedy", C.c_int),
                ("greedy_tol", C.c_double), ("mu_bar", C.c_void_p), ("history", C.c_void_p),
                ("max_history", C.c_int), ("n_history", C.c_void_p), ("pca_eps", C.c_double),
                ("prof_s", C.c_void_p)]


_lib = None


def library() -> C.CDLL:
    """Load liblrbms.so (built in-tree by paper_1405_2810_gb300.build)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_1405_2810_gb300.build.build()")
        lib = C.CDLL(LIB_PATH)
        vp, i, sz, dp = C.c_void_p, C.c_int, C.c_size_t, C.POINTER(C.c_double)
        lib.lrbms_create.argtypes = [C.POINTER(vp), C.POINTER(Config)]
        lib.lrbms_destroy.argtypes = [vp]
        lib.lrbms_offline_load.argtypes = [vp, C.POINTER(Problem), C.POINTER(Offline), C.POINTER(i)]
        lib.lrbms_offline_build.argtypes = [vp, i, C.POINTER(Problem), C.POINTER(BuildOpts), i,
                                            C.POINTER(vp), C.POINTER(i), C.POINTER(i)]
        lib.lrbms_clone.argtypes = [vp, i, vp, C.POINTER(i)]
        lib.lrbms_solve_noalloc.argtypes = [i, i, vp, vp, vp, vp, i, i, vp]
        lib.lrbms_step_io.argtypes = [vp, i, vp, i, C.POINTER(vp), C.POINTER(vp), vp]
        lib.lrbms_profile_start.argtypes = [vp, i]
        lib.lrbms_profile_read.argtypes = [vp, dp, dp, C.POINTER(i)]
        lib.lrbms_release.argtypes = [vp, i]
        lib.lrbms_step.argtypes = [vp, i, vp, i, vp]
        lib.lrbms_fine_step.argtypes = [vp, i, vp, i, vp]
        lib.lrbms_step_status.argtypes = [vp, i, vp]
        lib.lrbms_test_withhold_copy.argtypes = [vp, i]
        lib.lrbms_test_factor_plan.argtypes = [i, i, i, vp, vp]
        lib.lrbms_tuned_threads.argtypes = [vp, i, vp, C.POINTER(i), C.POINTER(i)]
        lib.lrbms_run.argtypes = [vp, i, i, vp, vp, vp]
        lib.lrbms_get_state.argtypes = [vp, i, vp, dp, dp]
        lib.lrbms_set_saturation.argtypes = [vp, i, vp]
        lib.lrbms_set_slopes.argtypes = [vp, i, vp]
        lib.lrbms_get_field.argtypes = [vp, i, i, vp, sz]
        lib.lrbms_field_bytes.argtypes = [vp, i, i]
        lib.lrbms_field_bytes.restype = sz
        lib.lrbms_sync.argtypes = [vp]
        lib.lrbms_memory.argtypes = [vp, C.POINTER(sz), C.POINTER(sz)]
        lib.lrbms_launch_count.argtypes = [vp]
        lib.lrbms_launch_count.restype = C.c_longlong
        lib.lrbms_last_error.argtypes = [vp]
        lib.lrbms_last_error.restype = C.c_char_p
        _lib = lib
    return _lib


def _ptr(a) -> int | None:
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    if not a.flags["C_CONTIGUOUS"]:
        raise ValueError("arrays passed to lrbms must be C-contiguous")
    return a.ctypes.data


def _check(ctx, rc):
    if rc != LRBMS_OK:
        msg = library().lrbms_last_error(ctx).decode() if ctx else ""
        raise LrbmsError(rc, msg)


def _as(a, dtype):
    if a is None or hasattr(a, "data_ptr"):
        return a
    return np.ascontiguousarray(a, dtype=dtype)


# ------------------------------------------------------------------ C-ABI names
def lrbms_create(precision=LRBMS_FP64, max_slots=64, hbm_budget=8 << 30, stream=None, device=0,
                 solver=LRBMS_SOLVE_FP64, refine_iters=0, refactor_period=0, refactor_stages=0):
    cfg = Config(precision, max_slots, hbm_budget, stream, device, solver, refine_iters, refactor_period,
                 refactor_stages)
    h = C.c_void_p()
    _check(None, library().lrbms_create(C.byref(h), C.byref(cfg)))
    return h


def lrbms_destroy(ctx):
    _check(ctx, library().lrbms_destroy(ctx))


def _problem_struct(problem: dict, keep: dict) -> Problem:
    pa = {k: _as(problem[k], dt) for k, dt in (("perm", np.float64), ("poro", np.float64),
                                             ("bc_type", np.int8), ("p_D", np.float64),
                                             ("v_N", np.float64), ("s_D", np.float64),
                                             ("s0", np.float64))}
    keep[id(pa)] = pa
    return Problem(problem["nx"], problem["ny"], problem["Sx"], problem["Sy"], problem["Lx"], problem["Ly"],
                   _ptr(pa["perm"]), _ptr(pa["poro"]), problem["eta_w"], problem["eta_o"],
                   problem.get("relperm", LRBMS_COREY), _ptr(pa["bc_type"]), _ptr(pa["p_D"]),
                   _ptr(pa["v_N"]), _ptr(pa["s_D"]), _ptr(pa["s0"]), problem.get("cfl", 0.5),
                   problem.get("dt_mode", LRBMS_DT_CFL), problem.get("dt_fixed", 0.0),
                   problem.get("dt_max", 0.0), problem.get("mean_weights", 0), problem.get("velocity", 0),
                   problem.get("transport", 0))


def lrbms_offline_build(ctx, problems, opts, n_copies: int = 1, rot=None, return_sizes=False):
    """Build offline data on the GPU for each problem (dicts as for
    lrbms_offline_load; opts: dicts with M, n_steps_T, N_E, mu, c_pen and
    optionally allow_fewer, greedy, greedy_tol, mu_bar, history, n_history,
    pca_eps, prof_s) and
    admit n_copies simulations per problem. rot: optional list (len
    n_prob*n_copies) of concatenated per-subdomain orthogonal matrices or
    None entries. Returns the simulation ids."""
    keep = {}
    n = len(problems)
    probs = (Problem * n)(*[_problem_struct(p, keep) for p in problems])
    ol = []
    for o in opts:
        ne = np.ascontiguousarray(o["N_E"], dtype=np.int32)
        mu = np.ascontiguousarray(o["mu"], dtype=np.float64)
        keep[id(ne)] = ne
        keep[id(mu)] = mu
        mub = None if o.get("mu_bar") is None else np.ascontiguousarray(o["mu_bar"], dtype=np.float64)
        hist = o.get("history")  # a float64 NumPy array to fill, or None
        nh = o.get("n_history")  # a one-element int32 NumPy array, or None
        keep[id(mub)] = mub
        ps = None if o.get("prof_s") is None else _as(o["prof_s"], np.float64)
        keep[id(ps)] = ps
        ol.append(BuildOpts(o["M"], o["n_steps_T"], _ptr(ne), mu.shape[0], _ptr(mu), o["c_pen"],
                            int(o.get("allow_fewer", 0)), int(o.get("greedy", 0)), float(o.get("greedy_tol", 0.0)),
                            _ptr(mub), _ptr(hist), 0 if hist is None else len(hist), _ptr(nh),
                            float(o.get("pca_eps", 0.0)), _ptr(ps)))
    oarr = (BuildOpts * n)(*ol)
    rp = None
    if rot is not None:
        rot = [None if r is None else np.ascontiguousarray(r, dtype=np.float64) for r in rot]
        keep["rot"] = rot
        rp = (C.c_void_p * len(rot))(*[None if r is None else _ptr(r) for r in rot])
    ids = (C.c_int * (n * n_copies))()
    n_sub = problems[0]["Sx"] * problems[0]["Sy"]
    got = (C.c_int * (n * n_sub))()
    _check(ctx, library().lrbms_offline_build(ctx, n, probs, oarr, n_copies, rp, ids, got))
    del keep
    if return_sizes:
        return list(ids), np.array(got, dtype=np.int32).reshape(n, n_sub)
    return list(ids)


def lrbms_clone(ctx, src: int, rot=None) -> int:
    """Admit a copy of simulation src with local bases rotated by rot
    (concatenated per-subdomain orthogonal matrices) or unrotated."""
    r = _as(rot, np.float64)
    sid = C.c_int()
    _check(ctx, library().lrbms_clone(ctx, src, _ptr(r), C.byref(sid)))
    return sid.value


def lrbms_offline_load(ctx, problem: dict, offline: dict) -> int:
    """problem/offline: dicts with the fields of lrbms_problem / lrbms_offline
    (arrays as NumPy arrays or device tensors)."""
    keep = {}
    pa = {k: _as(problem[k], dt) for k, dt in (("perm", np.float64), ("poro", np.float64),
                                             ("bc_type", np.int8), ("p_D", np.float64),
                                             ("v_N", np.float64), ("s_D", np.float64),
                                             ("s0", np.float64))}
    keep.update(pa)
    pr = Problem(problem["nx"], problem["ny"], problem["Sx"], problem["Sy"], problem["Lx"], problem["Ly"],
                 _ptr(pa["perm"]), _ptr(pa["poro"]), problem["eta_w"], problem["eta_o"],
                 problem.get("relperm", LRBMS_COREY), _ptr(pa["bc_type"]), _ptr(pa["p_D"]),
                 _ptr(pa["v_N"]), _ptr(pa["s_D"]), _ptr(pa["s0"]), problem.get("cfl", 0.5),
                 problem.get("dt_mode", LRBMS_DT_CFL), problem.get("dt_fixed", 0.0),
                 problem.get("dt_max", 0.0), problem.get("mean_weights", 0), problem.get("velocity", 0),
                   problem.get("transport", 0))
    oa = {k: _as(offline.get(k), dt) for k, dt in (("N_E", np.int32), ("prof_idx", np.uint8),
                                                 ("prof", np.float64), ("Gpinv", np.float64),
                                                 ("Phi", np.float64), ("Dblk", np.float64),
                                                 ("Fblk", np.float64), ("rhs", np.float64))}
    keep.update(oa)
    off = Offline(offline["M"], _ptr(oa["N_E"]), _ptr(oa["prof_idx"]), _ptr(oa["prof"]), _ptr(oa["Gpinv"]),
                  _ptr(oa["Phi"]), _ptr(oa["Dblk"]), _ptr(oa["Fblk"]), _ptr(oa["rhs"]),
                  offline["c_pen"], offline["Lf"])
    sid = C.c_int()
    _check(ctx, library().lrbms_offline_load(ctx, C.byref(pr), C.byref(off), C.byref(sid)))
    del keep
    return sid.value


def lrbms_release(ctx, sim_id: int):
    _check(ctx, library().lrbms_release(ctx, sim_id))


def lrbms_step(ctx, sim_ids, n_steps: int = 1, wait: bool = True):
    ids = np.ascontiguousarray(sim_ids, dtype=np.int32)
    status = np.zeros(len(ids), dtype=np.int32) if wait else None
    _check(ctx, library().lrbms_step(ctx, len(ids), _ptr(ids), n_steps, _ptr(status)))
    return status


def lrbms_fine_step(ctx, sim_ids, n_steps: int = 1):
    """Steps of the high-dimensional scheme (Algorithm 1) on resident
    simulations; returns the per-simulation status."""
    ids = np.ascontiguousarray(sim_ids, dtype=np.int32)
    status = np.zeros(len(ids), dtype=np.int32)
    _check(ctx, library().lrbms_fine_step(ctx, len(ids), _ptr(ids), n_steps, _ptr(status)))
    return status


def lrbms_step_status(ctx, n_sims: int):
    """Wait for the last lrbms_step(..., wait=False) and return its statuses."""
    status = np.zeros(n_sims, dtype=np.int32)
    _check(ctx, library().lrbms_step_status(ctx, n_sims, _ptr(status)))
    return status


N_PHASES = 7
PHASES = ["fit", "assemble", "solve", "reconstruct", "flux", "transport", "finalize"]


def lrbms_step_io(ctx, sim_ids, n_steps: int, s_in=None, s_out=None):
    """Step with the saturation exchanged with caller memory: s_in / s_out are
    lists of pinned host (or device) buffers, one per simulation."""
    ids = np.ascontiguousarray(sim_ids, dtype=np.int32)
    n = len(ids)
    pin = (C.c_void_p * n)(*[_ptr(a) for a in s_in]) if s_in is not None else None
    pout = (C.c_void_p * n)(*[_ptr(a) for a in s_out]) if s_out is not None else None
    status = np.zeros(n, dtype=np.int32)
    _check(ctx, library().lrbms_step_io(ctx, n, _ptr(ids), n_steps, pin, pout, _ptr(status)))
    return status


def lrbms_profile_start(ctx, max_steps: int):
    _check(ctx, library().lrbms_profile_start(ctx, max_steps))


def lrbms_profile_read(ctx, max_steps: int):
    """Returns (mean ms per phase [N_PHASES], ms per recorded step)."""
    ph = np.zeros(N_PHASES)
    st = np.zeros(max(max_steps, 1))
    n = C.c_int()
    _check(ctx, library().lrbms_profile_read(ctx, ph.ctypes.data_as(C.POINTER(C.c_double)),
                                             st.ctypes.data_as(C.POINTER(C.c_double)), C.byref(n)))
    return ph, st[: n.value]


def lrbms_run(ctx, sim_id: int, n_steps: int, s_out=None, p_out=None, flux_out=None):
    _check(ctx, library().lrbms_run(ctx, sim_id, n_steps, _ptr(s_out), _ptr(p_out), _ptr(flux_out)))


def lrbms_get_state(ctx, sim_id: int, s_out=None):
    t, m = C.c_double(), C.c_double()
    _check(ctx, library().lrbms_get_state(ctx, sim_id, _ptr(s_out), C.byref(t), C.byref(m)))
    return t.value, m.value


def lrbms_tuned_threads(ctx, sim_ids):
    """(assemble, reconstruct) CTA sizes the autotuner chose for these simulations."""
    ids = np.ascontiguousarray(sim_ids, dtype=np.int32)
    a, r = C.c_int(), C.c_int()
    _check(ctx, library().lrbms_tuned_threads(ctx, len(ids), _ptr(ids), C.byref(a), C.byref(r)))
    return a.value, r.value


def lrbms_test_withhold_copy(ctx, sim_id: int):
    """Test hook: the next reduced solve of sim_id withholds one bulk copy, so
    its bounded wait runs out and the simulation stops with LRBMS_E_TIMEOUT."""
    _check(ctx, library().lrbms_test_withhold_copy(ctx, sim_id))


def lrbms_test_factor_plan(n_sub: int, refactor_period: int, refactor_stages: int, info) -> tuple:
    """Test hook (host only): the factor kernel's plan for one step, as
    (k0, k1, buffer, whole, last_stage), from the solver state info[12]."""
    inf = np.ascontiguousarray(info, dtype=np.int32)
    assert inf.size == 12
    out = np.zeros(5, dtype=np.int32)
    _check(None, library().lrbms_test_factor_plan(n_sub, refactor_period, refactor_stages, _ptr(inf), _ptr(out)))
    return int(out[0]), int(out[1]), int(out[2]), bool(out[3]), bool(out[4])


def lrbms_set_slopes(ctx, sim_id: int, slopes):
    """Slopes [2][n_cells] of a simulation with the P1-DG transport."""
    sl = _as(slopes, np.float64)
    _check(ctx, library().lrbms_set_slopes(ctx, sim_id, _ptr(sl)))


def lrbms_set_saturation(ctx, sim_id: int, s):
    s = _as(s, np.float64)
    _check(ctx, library().lrbms_set_saturation(ctx, sim_id, _ptr(s)))


def lrbms_field_bytes(ctx, sim_id: int, field: int) -> int:
    return int(library().lrbms_field_bytes(ctx, sim_id, field))


def lrbms_get_field(ctx, sim_id: int, field: int, dtype=np.float64):
    nb = lrbms_field_bytes(ctx, sim_id, field)
    if nb == 0:
        raise LrbmsError(LRBMS_E_ARG, "unknown field or simulation")
    out = np.empty(nb // np.dtype(dtype).itemsize, dtype=dtype)
    _check(ctx, library().lrbms_get_field(ctx, sim_id, field, _ptr(out), nb))
    return out


def noalloc_sizes(Sx: int, Sy: int, N_E) -> tuple:
    """Element counts of the assembled blocks (per subdomain N_E^2, then per
    coarse face N_E- N_E+) and of the reduced vectors, for basis sizes N_E."""
    ne = np.asarray(N_E, dtype=np.int64).reshape(Sy, Sx)
    a = int(np.sum(ne * ne)) + int(np.sum(ne[:, :-1] * ne[:, 1:])) + int(np.sum(ne[:-1, :] * ne[1:, :]))
    return a, int(ne.sum())


def _device_f64(t, n: int) -> bool:
    return (hasattr(t, "data_ptr") and getattr(t, "is_cuda", False) and str(t.dtype) == "torch.float64"
            and t.is_contiguous() and t.numel() == n)


def lrbms_solve_noalloc(Sx: int, Sy: int, N_E, A, rhs, x, solver=LRBMS_SOLVE_FP64, refine_iters=0,
                        stream=None) -> int:
    """Solve an assembled reduced system with no allocation. A, rhs, x: CUDA
    float64 contiguous tensors of exactly the sizes the basis sizes give
    (noalloc_sizes); N_E: host int32 [Sx*Sy]. Returns the status code
    (LRBMS_E_ARG, without calling the library, for any other argument)."""
    ne = np.ascontiguousarray(N_E, dtype=np.int32)
    if Sx < 1 or Sy < 1 or ne.size != Sx * Sy:
        return LRBMS_E_ARG
    n_a, n = noalloc_sizes(Sx, Sy, ne)
    if not (_device_f64(A, n_a) and _device_f64(rhs, n) and _device_f64(x, n)):
        return LRBMS_E_ARG
    return int(library().lrbms_solve_noalloc(Sx, Sy, _ptr(ne), _ptr(A), _ptr(rhs), _ptr(x), solver,
                                             refine_iters, stream))


def lrbms_sync(ctx):
    _check(ctx, library().lrbms_sync(ctx))


def lrbms_memory(ctx):
    u, c = C.c_size_t(), C.c_size_t()
    _check(ctx, library().lrbms_memory(ctx, C.byref(u), C.byref(c)))
    return u.value, c.value


def lrbms_launch_count(ctx) -> int:
    return int(library().lrbms_launch_count(ctx))


def lrbms_last_error(ctx) -> str:
    return library().lrbms_last_error(ctx).decode()
