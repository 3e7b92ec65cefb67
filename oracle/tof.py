"""Time-of-flight (Section 3.5, Eq. timeOfFlight) for piecewise constants.

With a constant test function on cell e the volume term vanishes and the
equation reads sum_{f in de} tau^up_f F_f^{out,e} = phi_e |e|, where tau^up is
tau_e on faces the flux leaves e through, the neighbour's tau on faces it
enters through, and 0 on inflow boundary faces. The paper solves this
lower-block-triangular system by sweeping cells in flow order; the same
linear system is solved here with a sparse direct solver, which gives the
same unique solution for any ordering.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .grid import Grid


def time_of_flight(grid: Grid, F: np.ndarray, poro: np.ndarray) -> np.ndarray:
    n = grid.n_cells
    rows, cols, vals = [], [], []
    diag = np.zeros(n)
    f = grid.interior
    e1, e2 = grid.fe1[f], grid.fe2[f]
    Ff = F[f]
    # flux leaving e1 (F >= 0): contributes F tau_e1 to e1's row, and -F tau_e1 (inflow) to e2's row
    pos = Ff >= 0.0
    np.add.at(diag, e1[pos], Ff[pos])
    rows.append(e2[pos]); cols.append(e1[pos]); vals.append(-Ff[pos])
    neg = ~pos
    np.add.at(diag, e2[neg], -Ff[neg])
    rows.append(e1[neg]); cols.append(e2[neg]); vals.append(Ff[neg])
    Fout = F[grid.bface] * grid.bsign
    ob = Fout >= 0.0
    np.add.at(diag, grid.bcell[ob], Fout[ob])
    # guard cells without outflow (stagnant): a tiny diagonal keeps the system solvable
    tiny = 1e-300
    diag = np.where(diag > 0.0, diag, tiny)
    rows.append(np.arange(n)); cols.append(np.arange(n)); vals.append(diag)
    T = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n)).tocsc()
    return spla.spsolve(T, poro * grid.vol)
