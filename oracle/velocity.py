"""Conservative total-velocity reconstruction (Definition 2, Eq. velocityDG).

For a P1 pressure p and per-cell total mobility gamma = lambda(s), with
gravity G = 0, the normal flux through each face is

  int_f u . n = int_f ( -n . {gamma kappa grad p} + sigma_f/h_f [p]* ) ds

with [p]* = [p] on interior faces, p|Omega - p_D on Dirichlet faces (n
outward). On Neumann faces the boundary condition fixes the outward flux to
int_f v_N (reading R2: this is what makes the reconstruction locally
conservative; the discrete pressure equation tested with the indicator of a
cell gives exactly sum of outward fluxes = 0).

Returned fluxes are oriented along +x / +y for every face (interior and
boundary); a boundary face's outward flux is flux * outward sign.
The mean weights and penalty are those of ``swip``.
"""
from __future__ import annotations

import numpy as np

from .grid import Grid
from .swip import face_penalty, mean_weights, _normals


def face_fluxes(grid: Grid, perm: np.ndarray, gamma: np.ndarray, c_pen: float,
                bc_type: np.ndarray, p_D: np.ndarray, v_N: np.ndarray,
                p: np.ndarray, swapped: bool = False) -> np.ndarray:
    P = p.reshape(grid.n_cells, 3)
    Gr = grid.basis_gradients()
    grad = P @ Gr  # (n_cells, 2): grad p_e
    sig = face_penalty(grid, perm, c_pen)
    F = np.zeros(grid.n_faces)

    f = grid.interior
    e1, e2 = grid.fe1[f], grid.fe2[f]
    n = _normals(grid, f)
    t1, t2 = mean_weights(perm, e1, e2, swapped)
    mean_flux = (t1 * gamma[e1] * perm[e1]) * np.einsum("fd,fd->f", grad[e1], n) \
        + (t2 * gamma[e2] * perm[e2]) * np.einsum("fd,fd->f", grad[e2], n)
    pts, wq = grid.face_quadrature(f)
    v1 = grid.basis_values(e1[:, None], pts[..., 0], pts[..., 1])
    v2 = grid.basis_values(e2[:, None], pts[..., 0], pts[..., 1])
    jump = np.einsum("fqk,fk->fq", v1, P[e1]) - np.einsum("fqk,fk->fq", v2, P[e2])
    F[f] = np.einsum("fq,fq->f", wq, -mean_flux[:, None] + (sig[f] / grid.flen[f])[:, None] * jump)

    dsel = np.nonzero(bc_type == 1)[0]
    if len(dsel):
        fb = grid.bface[dsel]
        cb = grid.bcell[dsel]
        n = _normals(grid, fb, grid.bsign[dsel])
        flux_n = gamma[cb] * perm[cb] * np.einsum("fd,fd->f", grad[cb], n)
        pts, wq = grid.face_quadrature(fb)
        v = grid.basis_values(cb[:, None], pts[..., 0], pts[..., 1])
        jump = np.einsum("fqk,fk->fq", v, P[cb]) - p_D[dsel][:, None]
        Fout = np.einsum("fq,fq->f", wq, -flux_n[:, None] + (sig[fb] / grid.flen[fb])[:, None] * jump)
        F[fb] = Fout * grid.bsign[dsel]
    nsel = np.nonzero(bc_type == 0)[0]
    if len(nsel):
        fb = grid.bface[nsel]
        F[fb] = grid.flen[fb] * v_N[nsel] * grid.bsign[nsel]
    return F


def cell_outflows(grid: Grid, F: np.ndarray) -> np.ndarray:
    """Per cell, sum over its faces of the outward flux (the discrete
    divergence times |e|)."""
    out = np.zeros(grid.n_cells)
    f = grid.interior
    np.add.at(out, grid.fe1[f], F[f])
    np.add.at(out, grid.fe2[f], -F[f])
    np.add.at(out, grid.bcell, F[grid.bface] * grid.bsign)
    return out
