"""LRBMS offline phase: mobility profiles, least-squares fit, local bases and
the offline/online decomposition.

* Profiles (Algorithm 2, step 1(c)): Lambda^1 = lambda(0), Lambda^M = lambda(1)
  and, for q = 2..M-1, Lambda^q = lambda(0) where tau > (q-1) T/(M-2), else
  lambda(1) (total mobility; reading R8: piecewise constant, thresholding the
  cell value of the time-of-flight, T = n_steps * dt0 with dt0 the CFL step
  of the initial velocity).
* Fit (Eq. leastSquaresFit): Theta(s) = argmin || lambda(s) - sum theta_q
  Lambda^q ||_l2 over cell values, solved through the normal equations with
  the minimum-norm pseudo-inverse of G = P P^T (reading R6: eigen-decomposition,
  eigenvalues below 1e-12 * max dropped).
* Local bases (Algorithm 2, step 2): a greedy loop over a training set with
  the true energy error of Section 6 as error measure, extending each
  subdomain's basis by the Gram-Schmidt orthonormalised restriction of the
  worst-approximated snapshot (L2(E) inner product, two passes, rejection below
  1e-10 of the snapshot's local norm; reading R14). The constant function of
  every subdomain is the first basis function (reading R16). A plain
  snapshot variant (fixed random parameters, then truncation to given local
  sizes) serves the batched workloads.
* Components (Section 4.4): b_q = Phi^T K_vc(Lambda^q) Phi (volume and
  consistency terms), c = Phi^T K_pen Phi (penalty), d_q = Phi^T l_dc(Lambda^q)
  (Dirichlet consistency term), e = Phi^T (l_dp + l_neu) (Dirichlet penalty and
  Neumann terms); online, (c + sum theta_q b_q) p = e + sum theta_q d_q
  (Eq. reducedSystem).

A basis is kept per subdomain E as an array (3 n_E, N_E) whose row 3 c + k is
local basis function k of the c-th cell of ``Coarse.local_cell_order(E)``.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .grid import Grid, Coarse
from .impes import FineModel
from .physics import total_mobility
from .swip import bilinear, linear
from .tof import time_of_flight
from .transport import cfl_dt


# ---------------------------------------------------------------- profiles / fit
def profiles_from_tof(tau: np.ndarray, T: float, M: int, lam0: float, lam1: float):
    """Dense total-mobility profiles (M, n_cells) and, per cell, the first
    (1-based) profile index whose value is lambda(1)."""
    n = len(tau)
    P = np.empty((M, n))
    P[0] = lam0
    P[M - 1] = lam1
    for q in range(2, M):
        P[q - 1] = np.where(tau > (q - 1) * T / (M - 2), lam0, lam1)
    is1 = P == lam1
    if lam0 == lam1:
        k = np.full(n, M)
    else:
        k = np.argmax(is1, axis=0) + 1
    return P, k.astype(np.uint8)


def gram_pinv(P: np.ndarray, rcut: float = 1e-12) -> np.ndarray:
    """Minimum-norm pseudo-inverse of G = P P^T (symmetric eigen-decomposition)."""
    G = P @ P.T
    w, V = np.linalg.eigh(G)
    keep = w > rcut * w.max()
    inv = np.zeros_like(w)
    inv[keep] = 1.0 / w[keep]
    return (V * inv) @ V.T


def fit_theta(s, P, Gp, eta_w, eta_o, law):
    lam = total_mobility(s, eta_w, eta_o, law)
    return Gp @ (P @ lam)


# ---------------------------------------------------------------- local spaces
def local_mass_rows(grid: Grid, n_cells_E: int) -> np.ndarray:
    return np.tile(grid.local_mass(), n_cells_E)


def restrict(coarse: Coarse, p: np.ndarray, E: int) -> np.ndarray:
    cells = coarse.local_cell_order(E)
    return p.reshape(-1, 3)[cells].reshape(-1)


def orthonormalize(v: np.ndarray, basis: list, m: np.ndarray, reject_rtol: float = 1e-10):
    """Two-pass modified Gram-Schmidt of v against the columns in ``basis``
    with the L2(E) inner product (diagonal weights m). None if rejected."""
    n0 = np.sqrt(v @ (m * v))
    if n0 == 0.0:
        return None
    w = v.copy()
    for _ in range(2):
        for phi in basis:
            w = w - (phi @ (m * w)) * phi
    nw = np.sqrt(w @ (m * w))
    if nw < reject_rtol * n0:
        return None
    return w / nw


def unit_function(grid: Grid, n_cells_E: int) -> np.ndarray:
    v = np.zeros(3 * n_cells_E)
    v[0::3] = 1.0
    return v / np.sqrt(n_cells_E * grid.vol)


def global_basis(coarse: Coarse, Phi: list) -> sp.csr_matrix:
    """Sparse (3 n_cells, N) matrix whose columns are the local basis
    functions extended by zero (W_N subset of V_h, Section 4.2)."""
    rows, cols, vals = [], [], []
    off = 0
    for E, B in enumerate(Phi):
        cells = coarse.local_cell_order(E)
        dof = (3 * cells[:, None] + np.arange(3)[None, :]).reshape(-1)
        nE = B.shape[1]
        rows.append(np.repeat(dof, nE))
        cols.append(np.tile(np.arange(off, off + nE), len(dof)))
        vals.append(B.reshape(-1))
        off += nE
    nd = 3 * coarse.grid.n_cells
    return sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(nd, off)).tocsr()


# ---------------------------------------------------------------- fine operators
@dataclass
class FineOperators:
    """Parameter-independent fine pieces of Section 4.4."""
    K_vc: list            # per profile q: volume + consistency with Lambda^q
    K_pen: sp.csr_matrix  # penalty
    l_dc: list            # per profile q: Dirichlet consistency term with Lambda^q
    l_rest: np.ndarray    # Dirichlet penalty + Neumann terms


def fine_operators(model: FineModel, P: np.ndarray) -> FineOperators:
    g = model.grid
    ones = np.ones(g.n_cells)
    K_vc = [bilinear(g, model.perm, P[q], model.c_pen, model.bc_type, penalty=False,
                     swapped=model.swapped) for q in range(P.shape[0])]
    K_pen = bilinear(g, model.perm, ones, model.c_pen, model.bc_type, volume=False,
                     consistency=False, penalty=True, swapped=model.swapped)
    l_dc = [linear(g, model.perm, P[q], model.c_pen, model.bc_type, model.p_D, model.v_N,
                   dirichlet_penalty=False, dirichlet_consistency=True, neumann=False)
            for q in range(P.shape[0])]
    l_rest = linear(g, model.perm, ones, model.c_pen, model.bc_type, model.p_D, model.v_N,
                    dirichlet_penalty=True, dirichlet_consistency=False, neumann=True)
    return FineOperators(K_vc, K_pen, l_dc, l_rest)


def project(ops: FineOperators, Phi_g: sp.csr_matrix):
    """Reduced components (b_q, c, d_q, e) as dense arrays."""
    Pt = Phi_g.T.tocsr()
    B = np.stack([(Pt @ (K @ Phi_g)).toarray() for K in ops.K_vc])
    C = (Pt @ (ops.K_pen @ Phi_g)).toarray()
    d = np.stack([Pt @ l for l in ops.l_dc])
    e = Pt @ ops.l_rest
    return B, C, d, e


# ---------------------------------------------------------------- offline data
@dataclass
class Offline:
    M: int
    N_E: np.ndarray
    Phi: list
    B: np.ndarray
    C: np.ndarray
    d: np.ndarray
    e: np.ndarray
    P: np.ndarray
    prof_idx: np.ndarray
    Gp: np.ndarray
    c_pen: float
    Lf: float
    lam0: float
    lam1: float
    extra: dict = field(default_factory=dict)

    @property
    def N(self) -> int:
        return int(np.sum(self.N_E))

    @property
    def offsets(self) -> np.ndarray:
        return np.concatenate([[0], np.cumsum(self.N_E)]).astype(np.int64)


def initial_profiles(model: FineModel, s0: np.ndarray, n_steps: int, M: int):
    """Algorithm 2, step 1(a)-(c)."""
    lam = model.mobility(s0)
    p0 = model.solve_pressure(lam)
    F0 = model.fluxes(p0, lam)
    tau = time_of_flight(model.grid, F0, model.poro)
    dt0 = cfl_dt(model.grid, F0, model.poro, model.Lf, model.cfl)
    T = n_steps * dt0
    lam0 = float(total_mobility(0.0, model.eta_w, model.eta_o, model.law))
    lam1 = float(total_mobility(1.0, model.eta_w, model.eta_o, model.law))
    P, idx = profiles_from_tof(tau, T, M, lam0, lam1)
    return dict(p0=p0, F0=F0, tau=tau, T=T, P=P, idx=idx, lam0=lam0, lam1=lam1)


def saturation_profiles(model: FineModel, s0: np.ndarray, n_steps: int, M: int) -> np.ndarray:
    """Section 6 variant of Algorithm 2, step 1(c): the profiles are the
    mobilities of M high-dimensional saturations, Lambda^q = lambda(s_h^{n_q})
    (each phase's lambda_alpha^q = lambda_alpha(s_h^{n_q}), summed), taken
    along the fine scheme of Algorithm 1 started at s0. Reading: the paper
    does not space the times t^q; here n_q = round((q - 1) n_steps / (M - 1)),
    q = 1..M, so t^1 = 0 and t^M is the end of the n_steps-step run."""
    P = np.empty((M, model.grid.n_cells))
    s = np.array(s0, dtype=np.float64)
    n = 0
    for q in range(M):
        nq = int(round(q * n_steps / (M - 1)))
        while n < nq:
            s = model.step(s)["s"]
            n += 1
        P[q] = model.mobility(s)
    return P


def fine_solution(model: FineModel, P: np.ndarray, mu: np.ndarray) -> np.ndarray:
    """High-dimensional pressure for the mobility sum_q mu_q Lambda^q (Definition 1)."""
    return model.solve_pressure(mu @ P)


def greedy_bases(model: FineModel, coarse: Coarse, P: np.ndarray, ops: FineOperators,
                 train: np.ndarray, mu_bar: np.ndarray, cap: int, tol: float,
                 N_max: int = 10**9, max_iter: int = 200):
    """Algorithm 2, step 2 with the true energy error of Section 6."""
    g = model.grid
    nE = coarse.cx * coarse.cy
    m = local_mass_rows(g, nE)
    snaps = [fine_solution(model, P, mu) for mu in train]
    Kbar = bilinear(g, model.perm, mu_bar @ P, model.c_pen, model.bc_type, swapped=model.swapped)
    Phi = [[unit_function(g, nE)] for _ in range(coarse.n_sub)]
    history = []
    chosen = []  # training indices whose snapshots extended the bases
    for _ in range(max_iter):
        Phi_g = global_basis(coarse, [np.stack(b, axis=1) for b in Phi])
        B, C, d, e = project(ops, Phi_g)
        errs = np.empty(len(train))
        for t, mu in enumerate(train):
            A = C + np.tensordot(mu, B, axes=1)
            rhs = e + mu @ d
            x = sla.cho_solve(sla.cho_factor(A), rhs)
            diff = Phi_g @ x - snaps[t]
            errs[t] = np.sqrt(max(diff @ (Kbar @ diff), 0.0))
        k = int(np.argmax(errs))
        history.append(float(errs[k]))
        # step 2(g): go on only while |Xi| < N_max, here also while some
        # subdomain is below its cap (N_max read as the sum of the caps)
        if errs[k] <= tol or sum(len(b) for b in Phi) >= N_max or all(len(b) >= cap for b in Phi):
            break
        chosen.append(k)  # the snapshot set Psi of step 2(d)
        grew = False
        for E in range(coarse.n_sub):
            if len(Phi[E]) >= cap:
                continue
            w = orthonormalize(restrict(coarse, snaps[k], E), Phi[E], m)
            if w is not None:
                Phi[E].append(w)
                grew = True
        if not grew:
            break
    return [np.stack(b, axis=1) for b in Phi], history, chosen


def snapshot_bases(model: FineModel, coarse: Coarse, P: np.ndarray, mus: np.ndarray,
                   N_E: np.ndarray):
    """Unit function, then Gram-Schmidt of snapshots at the given parameters,
    truncated to N_E[E] functions per subdomain."""
    g = model.grid
    nE = coarse.cx * coarse.cy
    m = local_mass_rows(g, nE)
    snaps = [fine_solution(model, P, mu) for mu in mus]
    Phi = []
    for E in range(coarse.n_sub):
        b = [unit_function(g, nE)]
        for sn in snaps:
            if len(b) >= N_E[E]:
                break
            w = orthonormalize(restrict(coarse, sn, E), b, m)
            if w is not None:
                b.append(w)
        Phi.append(np.stack(b, axis=1))
    return Phi


def pca_bases(coarse: Coarse, snaps: list, grid: Grid, eps: float, max_size: int = 32):
    """Algorithm 2, step 3 (optional compression): on every subdomain E the
    principal components of the restrictions psi_1..psi_n of the selected
    snapshots, without centring (a proper orthogonal decomposition), in the
    L2(E) inner product. With the diagonal local mass m and the singular value
    decomposition sqrt(m) X = U diag(sigma) V^T (X = [psi_1 .. psi_n], sigma
    descending), the energies are l_k = sigma_k^2, the eigenvalues of the Gram
    matrix (psi_i, psi_j)_E; keep the fewest r modes whose discarded energy
    sum_{k > r} l_k is at most eps^2 sum_k l_k (r at most max_size), and
    phi_k = U e_k / sqrt(m) = sum_i V_ik psi_i / sigma_k, L2(E)-orthonormal.
    Singular values at most n eps_64 sigma_1 are round-off of a zero energy:
    they count as 0 and their modes are never kept.
    (Reading: the paper gives neither the criterion nor the tolerance.)"""
    nE = coarse.cx * coarse.cy
    m = local_mass_rows(grid, nE)
    sm = np.sqrt(m)
    Phi = []
    for E in range(coarse.n_sub):
        X = np.stack([restrict(coarse, sn, E) for sn in snaps], axis=1)  # (3 nE, n)
        U, sig, _ = np.linalg.svd(sm[:, None] * X, full_matrices=False)
        sig = np.where(sig > len(snaps) * np.finfo(float).eps * sig[0], sig, 0.0)
        lam = sig * sig
        total = lam.sum()
        tail = np.concatenate([np.cumsum(lam[::-1])[::-1][1:], [0.0]])  # tail[r-1] = sum_{k >= r} l_k (0-based)
        r = 1
        while r < len(lam) and r < max_size and lam[r] > 0.0 and tail[r - 1] > eps * eps * total:
            r += 1
        Phi.append(U[:, :r] / sm[:, None])
    return Phi


def build_offline(model: FineModel, coarse: Coarse, s0: np.ndarray, n_steps: int, M: int,
                  kind: str = "greedy", train=None, mu_bar=None, cap: int = 10,
                  tol: float = 1e-6, mus=None, N_E=None, Phi=None, P=None, pca_eps=None):
    """Algorithm 2 followed by the offline/online decomposition of Section
    4.4. With pca_eps set, the greedy's bases are replaced by the compression
    of step 3 (pca_bases) of the snapshots the greedy selected, at most cap
    modes per subdomain."""
    prof = initial_profiles(model, s0, n_steps, M)
    if P is None:
        P = prof["P"]
        idx = prof["idx"]
    else:
        idx = np.zeros(model.grid.n_cells, dtype=np.uint8)
    ops = fine_operators(model, P)
    hist = chosen = None
    if Phi is None:
        if kind == "greedy":
            if mu_bar is None:
                mu_bar = np.full(M, 1.0 / M)
            Phi, hist, chosen = greedy_bases(model, coarse, P, ops, train, mu_bar, cap, tol)
            if pca_eps is not None and chosen:
                snaps = [fine_solution(model, P, train[k]) for k in chosen]
                Phi = pca_bases(coarse, snaps, model.grid, pca_eps, max_size=cap)
        elif kind == "snapshots":
            Phi = snapshot_bases(model, coarse, P, mus, N_E)
        else:
            raise ValueError(kind)
    Phi_g = global_basis(coarse, Phi)
    B, C, d, e = project(ops, Phi_g)
    return Offline(M=M, N_E=np.array([b.shape[1] for b in Phi], dtype=np.int32), Phi=Phi,
                   B=B, C=C, d=d, e=e, P=P, prof_idx=idx, Gp=gram_pinv(P), c_pen=model.c_pen,
                   Lf=model.Lf, lam0=prof["lam0"], lam1=prof["lam1"],
                   extra=dict(tau=prof["tau"], T=prof["T"], p0=prof["p0"], greedy=hist,
                              chosen=chosen, ops=ops, Phi_g=Phi_g))
