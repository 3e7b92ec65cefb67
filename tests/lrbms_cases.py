"""Test cases for GPU-vs-oracle parity: seeded problems, the oracle's offline
phase, and the conversion of its offline data to the C-ABI layout of
include/lrbms.h (test infrastructure only)."""
from __future__ import annotations

import functools

import numpy as np

from oracle.grid import Coarse
from oracle.impes import FineModel
from oracle.offline import build_offline
from synth import make_problem, simplex_params, basis_sizes


def abi_problem(prob, model: FineModel, s0=None, dt_mode=0, dt_fixed=0.0, dt_max=0.0):
    return dict(nx=prob.nx, ny=prob.ny, Sx=prob.Sx, Sy=prob.Sy, Lx=prob.Lx, Ly=prob.Ly,
                perm=prob.perm, poro=prob.poro, eta_w=prob.eta_w, eta_o=prob.eta_o,
                relperm=0 if prob.relperm == "corey" else 1, bc_type=prob.bc_type,
                p_D=prob.p_D, v_N=prob.v_N, s_D=prob.s_D,
                s0=prob.s0 if s0 is None else s0, cfl=prob.cfl, dt_mode=dt_mode,
                dt_fixed=dt_fixed, dt_max=dt_max, mean_weights=1 if model.swapped else 0)


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


def rel(a, b) -> float:
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))
