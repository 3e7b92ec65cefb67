"""Fine Cartesian grid with face tables and the matching coarse grid.

Section 3.1: admissible tessellation, every face f has a unique normal n_f
pointing from e1 to e2, jump [w] = w|e1 - w|e2 and weighted mean
{w} = tau1 w|e1 + tau2 w|e2. Section 4.2: the coarse grid T_H must match the
fine grid (every coarse face is a union of fine faces); here the coarse cells
are Sx x Sy equal blocks of fine cells.

Numbering (shared with the library's documented layout):
  cell (i, j) -> j*nx + i
  x-faces (normal +x) (i, j), i = 0..nx, j = 0..ny-1  -> j*(nx+1) + i
  y-faces (normal +y) (i, j), i = 0..nx-1, j = 0..ny  -> nxf + j*nx + i
  boundary faces: left (j), right (j), bottom (i), top (i)
Interior face normals point to +x / +y; boundary faces use the outward normal.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class Grid:
    nx: int
    ny: int
    Lx: float
    Ly: float

    def __post_init__(self):
        self.hx = self.Lx / self.nx
        self.hy = self.Ly / self.ny
        self.n_cells = self.nx * self.ny
        self.vol = self.hx * self.hy
        i, j = np.meshgrid(np.arange(self.nx), np.arange(self.ny))
        self.ci = i.reshape(-1)
        self.cj = j.reshape(-1)
        self.xc = (self.ci + 0.5) * self.hx
        self.yc = (self.cj + 0.5) * self.hy
        self._build_faces()

    def cell(self, i, j):
        return j * self.nx + i

    def _build_faces(self):
        nx, ny = self.nx, self.ny
        nxf = (nx + 1) * ny
        nyf = nx * (ny + 1)
        self.nxf, self.nyf = nxf, nyf
        self.n_faces = nxf + nyf
        e1 = np.full(self.n_faces, -1, dtype=np.int64)
        e2 = np.full(self.n_faces, -1, dtype=np.int64)
        axis = np.zeros(self.n_faces, dtype=np.int64)
        mid = np.zeros((self.n_faces, 2))
        length = np.zeros(self.n_faces)
        for j in range(ny):
            for i in range(nx + 1):
                f = j * (nx + 1) + i
                axis[f] = 0
                if i > 0:
                    e1[f] = self.cell(i - 1, j)
                if i < nx:
                    e2[f] = self.cell(i, j)
                mid[f] = (i * self.hx, (j + 0.5) * self.hy)
                length[f] = self.hy
        for j in range(ny + 1):
            for i in range(nx):
                f = nxf + j * nx + i
                axis[f] = 1
                if j > 0:
                    e1[f] = self.cell(i, j - 1)
                if j < ny:
                    e2[f] = self.cell(i, j)
                mid[f] = ((i + 0.5) * self.hx, j * self.hy)
                length[f] = self.hx
        self.fe1, self.fe2, self.faxis, self.fmid, self.flen = e1, e2, axis, mid, length
        self.interior = np.nonzero((e1 >= 0) & (e2 >= 0))[0]
        # boundary faces in the documented order
        bf = []
        bout = []  # outward normal sign along the face axis
        for j in range(ny):
            bf.append(j * (nx + 1) + 0)
            bout.append(-1.0)
        for j in range(ny):
            bf.append(j * (nx + 1) + nx)
            bout.append(+1.0)
        for i in range(nx):
            bf.append(nxf + 0 * nx + i)
            bout.append(-1.0)
        for i in range(nx):
            bf.append(nxf + ny * nx + i)
            bout.append(+1.0)
        self.bface = np.array(bf, dtype=np.int64)
        self.bsign = np.array(bout)
        self.bcell = np.where(self.fe1[self.bface] >= 0, self.fe1[self.bface], self.fe2[self.bface])
        self.n_bfaces = len(bf)

    def face_normal(self, axis: int) -> np.ndarray:
        return np.array([1.0, 0.0]) if axis == 0 else np.array([0.0, 1.0])

    # P1 local basis on a rectangle: psi0 = 1, psi1 = 2(x-xc)/hx, psi2 = 2(y-yc)/hy
    # (the piecewise polynomial space V_h of Section 3.1 with k = 1).
    def basis_values(self, cells: np.ndarray, x: np.ndarray, y: np.ndarray) -> np.ndarray:
        v = np.empty(np.broadcast(cells, x).shape + (3,))
        v[..., 0] = 1.0
        v[..., 1] = 2.0 * (x - self.xc[cells]) / self.hx
        v[..., 2] = 2.0 * (y - self.yc[cells]) / self.hy
        return v

    def basis_gradients(self) -> np.ndarray:
        return np.array([[0.0, 0.0], [2.0 / self.hx, 0.0], [0.0, 2.0 / self.hy]])

    def local_mass(self) -> np.ndarray:
        """L2(e) Gram matrix of the local basis (diagonal: |e| (1, 1/3, 1/3))."""
        return self.vol * np.array([1.0, 1.0 / 3.0, 1.0 / 3.0])

    def face_quadrature(self, faces: np.ndarray):
        """Two-point Gauss rule on each face: points (nf, 2, 2) and weights (nf, 2)."""
        g = 0.5 / np.sqrt(3.0)
        mid = self.fmid[faces]
        ln = self.flen[faces]
        ax = self.faxis[faces]
        # tangential offset: along y for x-faces, along x for y-faces
        t = np.stack([ax == 1, ax == 0], axis=-1).astype(float)  # (nf, 2)
        pts = mid[:, None, :] + np.array([-g, g])[None, :, None] * ln[:, None, None] * t[:, None, :]
        w = np.repeat((0.5 * ln)[:, None], 2, axis=1)
        return pts, w


@dataclass
class Coarse:
    """Matching coarse grid of Sx x Sy subdomains (Section 4.2)."""
    grid: Grid
    Sx: int
    Sy: int

    def __post_init__(self):
        g = self.grid
        if g.nx % self.Sx or g.ny % self.Sy:
            raise ValueError("coarse grid must match the fine grid")
        self.cx = g.nx // self.Sx
        self.cy = g.ny // self.Sy
        self.n_sub = self.Sx * self.Sy
        self.sub_of_cell = (g.cj // self.cy) * self.Sx + (g.ci // self.cx)
        self.cells_of = [np.nonzero(self.sub_of_cell == E)[0] for E in range(self.n_sub)]
        # coarse faces: x-interfaces then y-interfaces, each as (E_minus, E_plus)
        cf = []
        for J in range(self.Sy):
            for I in range(self.Sx - 1):
                cf.append((J * self.Sx + I, J * self.Sx + I + 1))
        for J in range(self.Sy - 1):
            for I in range(self.Sx):
                cf.append((J * self.Sx + I, (J + 1) * self.Sx + I))
        self.cfaces = cf

    def local_cell_order(self, E: int) -> np.ndarray:
        """Fine cells of subdomain E in local lexicographic order (x fastest)."""
        I, J = E % self.Sx, E // self.Sx
        g = self.grid
        li, lj = np.meshgrid(np.arange(self.cx), np.arange(self.cy))
        return ((J * self.cy + lj) * g.nx + (I * self.cx + li)).reshape(-1)
