"""Test cases for GPU-vs-oracle parity: seeded problems, the oracle's offline
phase, and the conversion of its offline data to the C-ABI layout of
include/lrbms.h (test infrastructure only)."""
from __future__ import annotations

import functools

import numpy as np

from oracle.grid import Coarse
from oracle.impes import FineModel
from oracle.offline import (build_offline, initial_profiles, local_mass_rows, orthonormalize,
                            snapshot_bases)
from synth import make_problem, simplex_params, basis_sizes


def abi_problem(prob, model: FineModel, s0=None, dt_mode=0, dt_fixed=0.0, dt_max=0.0, velocity=0, transport=0):
    return dict(nx=prob.nx, ny=prob.ny, Sx=prob.Sx, Sy=prob.Sy, Lx=prob.Lx, Ly=prob.Ly,
                perm=prob.perm, poro=prob.poro, eta_w=prob.eta_w, eta_o=prob.eta_o,
                relperm=0 if prob.relperm == "corey" else 1, bc_type=prob.bc_type,
                p_D=prob.p_D, v_N=prob.v_N, s_D=prob.s_D,
                s0=prob.s0 if s0 is None else s0, cfl=prob.cfl, dt_mode=dt_mode,
                dt_fixed=dt_fixed, dt_max=dt_max, mean_weights=1 if model.swapped else 0, velocity=velocity,
                transport=transport)


def abi_offline(co: Coarse, off, dense_profiles: bool = False):
    offs = off.offsets
    n_sub = co.n_sub
    cells = co.cx * co.cy
    phi = []
    for E in range(n_sub):
        B = off.Phi[E]  # rows 3c+k
        nE = B.shape[1]
        phi.append(B.reshape(cells, 3, nE).transpose(2, 1, 0).reshape(-1))
    D, Fb, R = [], [], []
    for E in range(n_sub):
        sl = slice(offs[E], offs[E + 1])
        D.append(np.concatenate([off.C[sl, sl].reshape(-1)] + [off.B[q][sl, sl].reshape(-1) for q in range(off.M)]))
        R.append(np.concatenate([off.e[sl]] + [off.d[q][sl] for q in range(off.M)]))
    for (Em, Ep) in co.cfaces:
        sm = slice(offs[Em], offs[Em + 1])
        sp_ = slice(offs[Ep], offs[Ep + 1])
        Fb.append(np.concatenate([off.C[sm, sp_].reshape(-1)] + [off.B[q][sm, sp_].reshape(-1) for q in range(off.M)]))
    d = dict(M=off.M, N_E=off.N_E.astype(np.int32), Gpinv=off.Gp, Phi=np.concatenate(phi),
             Dblk=np.concatenate(D), Fblk=np.concatenate(Fb) if Fb else np.zeros(1), rhs=np.concatenate(R),
             c_pen=off.c_pen, Lf=off.Lf)
    if dense_profiles or not np.any(off.prof_idx):
        d["prof"] = np.ascontiguousarray(off.P)
        d["prof_idx"] = None
    else:
        d["prof_idx"] = off.prof_idx.astype(np.uint8)
        d["prof"] = None
    return d


def a_blocks(co: Coarse, off, A: np.ndarray) -> np.ndarray:
    """Dense reduced matrix -> the library's block layout (diagonal blocks, then
    coarse-face blocks)."""
    offs = off.offsets
    parts = [A[offs[E]:offs[E + 1], offs[E]:offs[E + 1]].reshape(-1) for E in range(co.n_sub)]
    for (Em, Ep) in co.cfaces:
        parts.append(A[offs[Em]:offs[Em + 1], offs[Ep]:offs[Ep + 1]].reshape(-1))
    return np.concatenate(parts)


@functools.lru_cache(maxsize=None)
def case(name: str, kind: str = "greedy", seed: int | None = None, swapped: bool = False, **kw):
    """(problem, fine model, coarse grid, oracle offline data) for a named case."""
    overrides = dict(kw)
    n = overrides.pop("n", None)
    S = overrides.pop("S", None)
    prob = make_problem(name, seed=seed, n=n, S=S, **overrides)
    m = FineModel.from_problem(prob, swapped=swapped)
    co = Coarse(m.grid, prob.Sx, prob.Sy)
    if kind == "greedy":
        off = build_offline(m, co, prob.s0, prob.n_steps, prob.M, kind="greedy",
                            train=simplex_params(32, prob.M, 11), cap=prob.n_max_local, tol=1e-6)
    else:
        NE = basis_sizes(co.n_sub, 3, min(12, 3 * co.cx * co.cy), prob.seed + 5)
        mus = simplex_params(int(NE.max()) + 2, prob.M, prob.seed + 6)
        off = build_offline(m, co, prob.s0, prob.n_steps, prob.M, kind="snapshots", mus=mus, N_E=NE)
    return prob, m, co, off


# Cases at the shapes the batched bench and the serving pool run: 8x8
# subdomains with basis sizes drawn from U{5..30} (both 16-row MMA tiles and
# all n-tiles of the FP32 factor), the same grid with sizes 17, 24, 30 and 32
# in neighbouring subdomains (residual rows above 16, the widest blocks), and
# 16x16 subdomains (the serving pool's widest envelope: 17 blocks per row).
SHAPES = {
    "bench-8x8": dict(n=64, S=8, lo=5, hi=30, seed=77),
    "bench-8x8-wide": dict(n=64, S=8, pattern=(17, 24, 30, 32), seed=78),
    "serve-16x16": dict(n=128, S=16, lo=5, hi=30, seed=79),
}


@functools.lru_cache(maxsize=None)
def shape_case(label: str):
    """(problem, fine model, coarse grid, oracle offline data) for one of
    SHAPES: the batched workload's physics (seeded log-normal field, Corey,
    viscosity ratio from U[2, 20]) with snapshot bases of the given sizes."""
    sp_ = SHAPES[label]
    prob = make_problem("batch", n=sp_["n"], S=sp_["S"], sim_index=sp_["seed"])
    m = FineModel.from_problem(prob)
    co = Coarse(m.grid, prob.Sx, prob.Sy)
    if "pattern" in sp_:
        pat = np.array(sp_["pattern"], dtype=np.int32)
        I = np.arange(co.n_sub) % prob.Sx
        J = np.arange(co.n_sub) // prob.Sx
        NE = pat[(I + 2 * J) % len(pat)]  # every x and y neighbour has another size
    else:
        NE = basis_sizes(co.n_sub, sp_["lo"], sp_["hi"], sp_["seed"] + 5)
    mus = simplex_params(int(NE.max()) + 4, prob.M, sp_["seed"] + 6)
    P = initial_profiles(m, prob.s0, prob.n_steps, prob.M)["P"]
    Phi = snapshot_bases(m, co, P, mus, NE)
    # Where the snapshots span fewer functions than asked (their restrictions
    # become dependent), top the basis up with seeded random P1 functions,
    # orthonormalised the same way: any local basis is a valid reduced space.
    rng = np.random.default_rng(np.random.PCG64(sp_["seed"] + 7))
    mloc = local_mass_rows(m.grid, co.cx * co.cy)
    for E in range(co.n_sub):
        cols = [Phi[E][:, i] for i in range(Phi[E].shape[1])]
        while len(cols) < NE[E]:
            w = orthonormalize(rng.standard_normal(3 * co.cx * co.cy), cols, mloc)
            if w is not None:
                cols.append(w)
        Phi[E] = np.stack(cols, axis=1)
    off = build_offline(m, co, prob.s0, prob.n_steps, prob.M, Phi=Phi)
    assert np.array_equal(off.N_E, NE)
    return prob, m, co, off


@functools.lru_cache(maxsize=None)
def shape_states(label: str, n_steps: int):
    """Oracle saturations s^0 .. s^n_steps of a SHAPES case (the reduced
    trajectory), for per-step parity from identical inputs."""
    from oracle.reduced import online_step
    prob, m, co, off = shape_case(label)
    out = [prob.s0.copy()]
    for _ in range(n_steps):
        out.append(online_step(m, off, out[-1])["s"])
    return tuple(out)


def close_elementwise(a, b, tol: float) -> float:
    """max_i |a_i - b_i| / max_i |b_i| (the element-wise counterpart of rel);
    callers assert it is at most tol."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    mb = np.abs(b).max() if b.size else 0.0
    return float(np.abs(a - b).max() / (mb if mb > 0 else 1.0)) if b.size else 0.0


def rel(a, b) -> float:
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))
