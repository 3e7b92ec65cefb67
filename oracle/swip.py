"""SWIP-DG pressure discretisation (Section 3.2), P1 on rectangles, FP64.

Bilinear form b_h(v, w; gamma) of Eq. swipBilP with the standard SWIP sign of
the consistency and symmetry terms (reading R1: the printed "+" is taken as
"-", matching the sign of the Dirichlet term of l_h and of Eq. velocityDG):

  b_h(v,w) =  sum_e  int_e gamma kappa grad v . grad w
            + sum_{f in Gi u Gd} sigma_f/h_f int_f [v][w]
            - sum_{f in Gi u Gd} int_f ({gamma kappa grad v . n}[w] + {gamma kappa grad w . n}[v])

Penalty (Eq. penaltyParam with Remark 1): sigma_f = c_pen * 2 a1 a2/(a1+a2),
a_l = kappa on side l, c_pen = c_f / max(eta_w, eta_o) (the mobility is kept
out of the penalty); on a boundary face sigma_f = c_pen * kappa_e. h_f is the
face diameter. Weighted mean (Section 3.1): {w} = tau1 w1 + tau2 w2 with
tau_l = a_l/(a1+a2) (reading R3, literal); ``swapped=True`` takes
tau1 = a2/(a1+a2), tau2 = a1/(a1+a2) instead. On a boundary face the mean is
the one-sided value, [w] = w and n is the outward normal.

Linear form l_h (Section 3.2) with q1 optional, gravity G = 0 and the
Neumann sign of reading R2 (the boundary condition prescribes the outward flux
-gamma kappa grad p . n = v_N, so the term enters as -int v_N w):

  l_h(w) = int q1 w + sum_{f in Gd} int_f (sigma_f/h_f w - gamma kappa grad w . n) p_D
           - sum_{f in Gn} int_f v_N w

Volume integrals of P1 products with a per-cell coefficient are exact
(|e| times the constant integrand); face integrals use the two-point Gauss
rule, exact for products of linears. Global dof of (cell e, local basis k) is
3*e + k with the local basis of ``Grid.basis_values``.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .grid import Grid


def face_penalty(grid: Grid, perm: np.ndarray, c_pen: float):
    """sigma_f per face (interior: harmonic form, boundary: one-sided)."""
    sig = np.zeros(grid.n_faces)
    f = grid.interior
    k1, k2 = perm[grid.fe1[f]], perm[grid.fe2[f]]
    sig[f] = c_pen * 2.0 * k1 * k2 / (k1 + k2)
    sig[grid.bface] = c_pen * perm[grid.bcell]
    return sig


def mean_weights(perm: np.ndarray, e1: np.ndarray, e2: np.ndarray, swapped: bool):
    k1, k2 = perm[e1], perm[e2]
    if swapped:
        return k2 / (k1 + k2), k1 / (k1 + k2)
    return k1 / (k1 + k2), k2 / (k1 + k2)


def _normals(grid: Grid, faces: np.ndarray, sign: np.ndarray | None = None) -> np.ndarray:
    n = np.zeros((len(faces), 2))
    ax = grid.faxis[faces]
    n[ax == 0, 0] = 1.0
    n[ax == 1, 1] = 1.0
    if sign is not None:
        n *= sign[:, None]
    return n


def bilinear(grid: Grid, perm: np.ndarray, gamma: np.ndarray, c_pen: float,
             bc_type: np.ndarray, *, volume: bool = True, consistency: bool = True,
             penalty: bool = True, swapped: bool = False) -> sp.csr_matrix:
    """Matrix K with K[row=w dof, col=v dof] = b_h(v, w; gamma) restricted to
    the selected terms. gamma is the per-cell total mobility."""
    nd = 3 * grid.n_cells
    rows, cols, vals = [], [], []
    Gr = grid.basis_gradients()  # (3, 2)

    if volume:
        # int_e gamma kappa grad psi_i . grad psi_j = gamma kappa |e| (Gr Gr^T)_ij
        loc = Gr @ Gr.T
        coef = gamma * perm * grid.vol
        e = np.arange(grid.n_cells)
        idx = 3 * e[:, None] + np.arange(3)[None, :]
        rows.append(np.repeat(idx[:, :, None], 3, axis=2).reshape(-1))
        cols.append(np.repeat(idx[:, None, :], 3, axis=1).reshape(-1))
        vals.append((coef[:, None, None] * loc[None]).reshape(-1))

    sig = face_penalty(grid, perm, c_pen)

    # interior faces
    f = grid.interior
    e1, e2 = grid.fe1[f], grid.fe2[f]
    pts, wq = grid.face_quadrature(f)
    v1 = grid.basis_values(e1[:, None], pts[..., 0], pts[..., 1])  # (nf, 2, 3)
    v2 = grid.basis_values(e2[:, None], pts[..., 0], pts[..., 1])
    n = _normals(grid, f)
    gn = n @ Gr.T  # (nf, 3): grad psi_k . n
    t1, t2 = mean_weights(perm, e1, e2, swapped)
    c1 = t1 * gamma[e1] * perm[e1]
    c2 = t2 * gamma[e2] * perm[e2]
    J = np.concatenate([v1, -v2], axis=2)  # jump of each of the 6 local functions
    Mn = np.concatenate([c1[:, None] * gn, c2[:, None] * gn], axis=1)  # mean flux
    loc = np.zeros((len(f), 6, 6))
    if penalty:
        ph = sig[f] / grid.flen[f]
        loc += np.einsum("fq,fqi,fqj->fij", wq * ph[:, None], J, J)
    if consistency:
        Jint = np.einsum("fq,fqi->fi", wq, J)  # int_f [psi]
        loc -= Jint[:, :, None] * Mn[:, None, :]   # -{k grad v.n}[w]: row w, col v
        loc -= Mn[:, :, None] * Jint[:, None, :]   # -{k grad w.n}[v]
    idx = np.concatenate([3 * e1[:, None] + np.arange(3), 3 * e2[:, None] + np.arange(3)], axis=1)
    rows.append(np.repeat(idx[:, :, None], 6, axis=2).reshape(-1))
    cols.append(np.repeat(idx[:, None, :], 6, axis=1).reshape(-1))
    vals.append(loc.reshape(-1))

    # Dirichlet boundary faces
    bsel = np.nonzero(bc_type == 1)[0]
    if len(bsel):
        fb = grid.bface[bsel]
        cb = grid.bcell[bsel]
        pts, wq = grid.face_quadrature(fb)
        v = grid.basis_values(cb[:, None], pts[..., 0], pts[..., 1])  # (nb, 2, 3)
        n = _normals(grid, fb, grid.bsign[bsel])
        gn = n @ Gr.T
        Mn = (gamma[cb] * perm[cb])[:, None] * gn
        loc = np.zeros((len(fb), 3, 3))
        if penalty:
            ph = sig[fb] / grid.flen[fb]
            loc += np.einsum("fq,fqi,fqj->fij", wq * ph[:, None], v, v)
        if consistency:
            Jint = np.einsum("fq,fqi->fi", wq, v)
            loc -= Jint[:, :, None] * Mn[:, None, :]
            loc -= Mn[:, :, None] * Jint[:, None, :]
        idx = 3 * cb[:, None] + np.arange(3)
        rows.append(np.repeat(idx[:, :, None], 3, axis=2).reshape(-1))
        cols.append(np.repeat(idx[:, None, :], 3, axis=1).reshape(-1))
        vals.append(loc.reshape(-1))

    K = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(nd, nd)).tocsr()
    K.sum_duplicates()
    return K


def linear(grid: Grid, perm: np.ndarray, gamma: np.ndarray, c_pen: float,
           bc_type: np.ndarray, p_D: np.ndarray, v_N: np.ndarray, *,
           dirichlet_penalty: bool = True, dirichlet_consistency: bool = True,
           neumann: bool = True, source=None) -> np.ndarray:
    """Vector l with l[w dof] = l_h(w) restricted to the selected terms.
    ``source`` is an optional callable q1(x, y) (2x2 Gauss per cell)."""
    nd = 3 * grid.n_cells
    out = np.zeros(nd)
    Gr = grid.basis_gradients()
    sig = face_penalty(grid, perm, c_pen)
    bsel = np.nonzero(bc_type == 1)[0]
    if len(bsel):
        fb = grid.bface[bsel]
        cb = grid.bcell[bsel]
        pts, wq = grid.face_quadrature(fb)
        v = grid.basis_values(cb[:, None], pts[..., 0], pts[..., 1])
        n = _normals(grid, fb, grid.bsign[bsel])
        gn = n @ Gr.T
        contrib = np.zeros((len(fb), 3))
        if dirichlet_penalty:
            ph = sig[fb] / grid.flen[fb]
            contrib += np.einsum("fq,fqi->fi", wq * ph[:, None], v) * p_D[bsel][:, None]
        if dirichlet_consistency:
            lk = gamma[cb] * perm[cb]
            contrib -= (wq.sum(axis=1) * lk * p_D[bsel])[:, None] * gn
        np.add.at(out, 3 * cb[:, None] + np.arange(3), contrib)
    nsel = np.nonzero(bc_type == 0)[0]
    if neumann and len(nsel):
        fb = grid.bface[nsel]
        cb = grid.bcell[nsel]
        pts, wq = grid.face_quadrature(fb)
        v = grid.basis_values(cb[:, None], pts[..., 0], pts[..., 1])
        contrib = -np.einsum("fq,fqi->fi", wq, v) * v_N[nsel][:, None]
        np.add.at(out, 3 * cb[:, None] + np.arange(3), contrib)
    if source is not None:
        g = 0.5 / np.sqrt(3.0)
        for ox in (-g, g):
            for oy in (-g, g):
                x = grid.xc + ox * grid.hx
                y = grid.yc + oy * grid.hy
                v = grid.basis_values(np.arange(grid.n_cells), x, y)
                out += (0.25 * grid.vol * source(x, y)[:, None] * v).reshape(-1)
    return out


def pressure_system(grid: Grid, perm, gamma, c_pen, bc_type, p_D, v_N, swapped=False, source=None):
    """Definition 1: b_h(p_h, w; gamma) = l_h(w) for all w in V_h."""
    K = bilinear(grid, perm, gamma, c_pen, bc_type, swapped=swapped)
    l = linear(grid, perm, gamma, c_pen, bc_type, p_D, v_N, source=source)
    return K, l


def default_penalty_scale(eta_w: float, eta_o: float, c_f: float | None = None) -> float:
    """c_pen = c_f / max(eta_w, eta_o) (Remark 1) with the default
    c_f = 20 max(eta)/min(eta) (reading R4), i.e. c_pen = 20 / min(eta)."""
    if c_f is None:
        c_f = 20.0 * max(eta_w, eta_o) / min(eta_w, eta_o)
    return c_f / max(eta_w, eta_o)
