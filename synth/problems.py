"""Seeded problem definitions for the two-phase workloads (pure data).

A ``Problem`` holds what the paper's model problem needs (Section 2,
Eqs. mainPressure..mainInitialData): a 2D Cartesian fine grid on
[0, Lx] x [0, Ly], a matching coarse grid of Sx x Sy subdomains (Section 4.2),
per-cell permeability and porosity, the two viscosities, the relative
permeability law, boundary data per boundary face and the initial saturation.

Boundary faces are numbered left side (bottom to top), right side (bottom to
top), bottom side (left to right), top side (left to right); there are
2*ny + 2*nx of them. Per boundary face: ``bc_type`` 1 = Dirichlet pressure
p_D, 0 = Neumann with prescribed outward flux density v_N (0 = no-flow);
``s_D`` is the saturation carried in when the face is an inflow face.

Workloads (seeded stand-ins; the paper's fields exist only as figures):
  small    32x32 fine, 4x4 subdomains, sigma=1 / corr 0.1 log-normal,
           viscosity ratio 10, Corey, 50 steps, <=10 basis functions/subdomain
  aniso    256x256 fine, 16x16 subdomains, corr (0.2, 0.02), contrast 1e6,
           viscosity ratio 5, 500 steps, <=20 basis functions/subdomain
  batch    128x128 fine, 8x8 subdomains, sigma=1 / corr 0.1, viscosity ratio
           U[2, 20] per simulation, basis sizes U{5..30} per subdomain
  served   grid n in {64,128,256,512}, subdomains S in {4,8,16,32}, n/S >= 4
  paper_bc the paper's benchmark boundary conditions (Section 6): Dirichlet
           inflow on the left (p = p_inflow, 10 in the paper), Neumann outflow
           v_N = 3e-4 on the right, no-flow top/bottom
  rect     nx x ny fine grid with Sx x Sy subdomains given as n=(nx, ny),
           S=(Sx, Sy) (sizes that leave ragged tiles)
  strip    n x 1 strip with Dirichlet pressure at both ends (1D transport)
All fields use porosity 0.2, eta_w = 1, eta_o = viscosity ratio, s0 = 0.
Default boundary conditions: left Dirichlet p = 1 with s_D = 1 (injection),
right Dirichlet p = 0, top and bottom no-flow.
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace

import numpy as np

from .fields import lognormal_field


@dataclass
class Problem:
    nx: int
    ny: int
    Lx: float
    Ly: float
    Sx: int
    Sy: int
    perm: np.ndarray
    poro: np.ndarray
    eta_w: float
    eta_o: float
    relperm: str  # "corey" (k_rw = s^2, k_ro = (1-s)^2) or "linear"
    bc_type: np.ndarray  # int8 per boundary face
    p_D: np.ndarray
    v_N: np.ndarray
    s_D: np.ndarray
    s0: np.ndarray
    n_steps: int = 50
    cfl: float = 0.5
    M: int = 8
    n_max_local: int = 10
    name: str = ""
    seed: int = 0
    extra: dict = field(default_factory=dict)

    @property
    def n_cells(self) -> int:
        return self.nx * self.ny

    @property
    def n_sub(self) -> int:
        return self.Sx * self.Sy

    def with_(self, **kw) -> "Problem":
        return replace(self, **kw)


def boundary_face_count(nx: int, ny: int) -> int:
    return 2 * ny + 2 * nx


def default_bcs(nx: int, ny: int, p_left: float = 1.0, p_right: float = 0.0,
                right: str = "dirichlet", v_out: float = 0.0):
    nb = boundary_face_count(nx, ny)
    bc_type = np.zeros(nb, dtype=np.int8)
    p_D = np.zeros(nb)
    v_N = np.zeros(nb)
    s_D = np.zeros(nb)
    left = slice(0, ny)
    rgt = slice(ny, 2 * ny)
    bc_type[left] = 1
    p_D[left] = p_left
    s_D[left] = 1.0
    if right == "dirichlet":
        bc_type[rgt] = 1
        p_D[rgt] = p_right
    else:
        bc_type[rgt] = 0
        v_N[rgt] = v_out
    return bc_type, p_D, v_N, s_D


def make_problem(name: str, seed: int | None = None, sim_index: int = 0,
                 n: int | None = None, S: int | None = None, p_inflow: float = 10.0,
                 **overrides) -> Problem:
    """Build one seeded workload by name (see module docstring)."""
    if name == "small":
        nx = ny = 32
        Sx = Sy = 4
        sd = 1405 if seed is None else seed
        perm = lognormal_field(nx, ny, 1.0, 1.0, 1.0, (0.1, 0.1), sd)
        ratio = 10.0
        steps, nmax = 50, 10
    elif name == "aniso":
        nx = ny = 256
        Sx = Sy = 16
        sd = 2810 if seed is None else seed
        perm = lognormal_field(nx, ny, 1.0, 1.0, 1.0, (0.2, 0.02), sd, contrast=1e6)
        ratio = 5.0
        steps, nmax = 500, 20
    elif name == "batch":
        nx = ny = 128 if n is None else n
        Sx = Sy = 8 if S is None else S
        sd = (7000 if seed is None else seed) + sim_index
        perm = lognormal_field(nx, ny, 1.0, 1.0, 1.0, (0.1, 0.1), sd)
        ratio = float(np.random.default_rng(np.random.PCG64(sd + 10**6)).uniform(2.0, 20.0))
        steps, nmax = 300, 30
    elif name == "served":
        nx = ny = 64 if n is None else n
        Sx = Sy = 4 if S is None else S
        if nx // Sx < 4:
            raise ValueError("served workload needs at least 4x4 fine cells per subdomain")
        sd = (9000 if seed is None else seed) + sim_index
        perm = lognormal_field(nx, ny, 1.0, 1.0, 1.0, (0.1, 0.1), sd)
        ratio = float(np.random.default_rng(np.random.PCG64(sd + 10**6)).uniform(2.0, 20.0))
        steps, nmax = 300, 30
    elif name == "paper_bc":
        nx = 40 if n is None else n
        ny = 16 if n is None else max(2, (2 * n) // 5)
        Sx, Sy = (4, 2) if S is None else (S, max(1, S // 2))
        sd = 1998 if seed is None else seed
        perm = lognormal_field(nx, ny, 300.0, 60.0, 1.0, (30.0, 6.0), sd)
        ratio = 0.008 / 0.00130581
        steps, nmax = 50, 10
    elif name == "rect":
        nx, ny = (48, 40) if n is None else n
        Sx, Sy = (4, 5) if S is None else S
        sd = 4242 if seed is None else seed
        perm = lognormal_field(nx, ny, 1.0, 1.0, 1.0, (0.1, 0.1), sd)
        ratio = 4.0
        steps, nmax = 20, 8
    elif name == "strip":
        nx = 64 if n is None else n
        ny = 1
        Sx, Sy = (4 if S is None else S), 1
        sd = 0 if seed is None else seed
        perm = np.ones(nx * ny)
        ratio = 2.0
        steps, nmax = 100, 10
    else:
        raise ValueError(f"unknown workload {name!r}")

    if name == "paper_bc":
        Lx, Ly = 300.0, 60.0
        bcs = default_bcs(nx, ny, p_left=p_inflow, right="neumann", v_out=3e-4)
        eta_w, eta_o = 0.00130581, 0.008
        relperm = "linear"
    else:
        Lx = Ly = 1.0
        if name == "strip":
            Lx, Ly = 1.0, 1.0 / nx
        bcs = default_bcs(nx, ny)
        eta_w, eta_o = 1.0, ratio
        relperm = "corey"
    bc_type, p_D, v_N, s_D = bcs
    prob = Problem(nx=nx, ny=ny, Lx=Lx, Ly=Ly, Sx=Sx, Sy=Sy, perm=perm,
                   poro=np.full(nx * ny, 0.2), eta_w=eta_w, eta_o=eta_o,
                   relperm=relperm, bc_type=bc_type, p_D=p_D, v_N=v_N, s_D=s_D,
                   s0=np.zeros(nx * ny), n_steps=steps, M=8, n_max_local=nmax,
                   name=name, seed=sd)
    if overrides:
        prob = prob.with_(**overrides)
    return prob


def simplex_params(n: int, M: int, seed: int, lo: float = 1e-4) -> np.ndarray:
    """n random parameters in [lo, 1]^M with unit sum (the paper's training
    set recipe, Section 6): lo + (1 - M lo) * Dirichlet(1, ..., 1)."""
    rng = np.random.default_rng(np.random.PCG64(seed))
    return lo + (1.0 - M * lo) * rng.dirichlet(np.ones(M), size=n)


def basis_sizes(n_sub: int, lo: int, hi: int, seed: int) -> np.ndarray:
    """Local basis sizes drawn uniformly from {lo..hi}."""
    rng = np.random.default_rng(np.random.PCG64(seed))
    return rng.integers(lo, hi + 1, size=n_sub).astype(np.int32)


def random_orthogonal(n: int, rng: np.random.Generator) -> np.ndarray:
    """Haar-distributed orthogonal n x n matrix (QR of a Gaussian matrix with
    the signs of R's diagonal moved into Q)."""
    a = rng.standard_normal((n, n))
    q, r = np.linalg.qr(a)
    return q * np.sign(np.diag(r))[None, :]
