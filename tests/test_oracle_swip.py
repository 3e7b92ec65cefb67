"""Pins for the oracle's SWIP-DG pressure discretisation and velocity
reconstruction (Section 3.2, Definition 1, Definition 2) against closed forms,
invariants and brute-force quadrature."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle.grid import Grid
from oracle.impes import FineModel
from oracle.swip import bilinear, linear, pressure_system
from oracle.velocity import face_fluxes, cell_outflows
from synth import make_problem
from synth.problems import default_bcs, boundary_face_count


def _solve(g, perm, gam, c_pen, bc, pD, vN, swapped=False, source=None):
    K, l = pressure_system(g, perm, gam, c_pen, bc, pD, vN, swapped=swapped, source=source)
    return spla.spsolve(K.tocsc(), l)


def test_local_basis_mass_matches_quadrature():
    g = Grid(3, 2, 1.5, 0.7)
    # 3x3 Gauss-Legendre per cell: exact for the quadratic integrands psi_i psi_j
    xg, wg = np.polynomial.legendre.leggauss(3)
    e = 4
    M = np.zeros((3, 3))
    for a, wa in zip(xg, wg):
        for b, wb in zip(xg, wg):
            x = g.xc[e] + 0.5 * g.hx * a
            y = g.yc[e] + 0.5 * g.hy * b
            v = g.basis_values(np.array([e]), np.array([x]), np.array([y]))[0]
            M += 0.25 * g.vol * wa * wb * np.outer(v, v)
    assert np.allclose(M, np.diag(g.local_mass()), atol=1e-15)


def test_swip_symmetric_and_spd():
    prob = make_problem("small")
    m = FineModel.from_problem(prob)
    rng = np.random.default_rng(3)
    gam = rng.uniform(m.mobility(0.0), m.mobility(1.0), m.grid.n_cells)
    K, _ = pressure_system(m.grid, m.perm, gam, m.c_pen, m.bc_type, m.p_D, m.v_N)
    Kd = K.toarray()
    assert np.abs(Kd - Kd.T).max() <= 1e-12 * np.abs(Kd).max()
    np.linalg.cholesky(Kd)  # raises if not SPD


@pytest.mark.parametrize("direction", ["x", "y"])
def test_linear_pressure_closed_form(direction):
    """T1: homogeneous kappa, constant mobility, Dirichlet p = 1 / p = 0 on two
    opposite sides, no-flow elsewhere: p = 1 - x (or 1 - y) on every dof."""
    n = 12
    g = Grid(n, n, 1.0, 1.0)
    nb = boundary_face_count(n, n)
    bc = np.zeros(nb, dtype=np.int8)
    pD = np.zeros(nb)
    if direction == "x":
        bc[0:n] = 1; pD[0:n] = 1.0; bc[n:2 * n] = 1
    else:
        bc[2 * n:3 * n] = 1; pD[2 * n:3 * n] = 1.0; bc[3 * n:4 * n] = 1
    perm = np.full(g.n_cells, 3.0)
    gam = np.full(g.n_cells, 0.7)
    p = _solve(g, perm, gam, 20.0, bc, pD, np.zeros(nb)).reshape(-1, 3)
    if direction == "x":
        exact = np.stack([1 - g.xc, np.full(g.n_cells, -g.hx / 2), np.zeros(g.n_cells)], 1)
    else:
        exact = np.stack([1 - g.yc, np.zeros(g.n_cells), np.full(g.n_cells, -g.hy / 2)], 1)
    assert np.abs(p - exact).max() < 1e-12
    F = face_fluxes(g, perm, gam, 20.0, bc, pD, np.zeros(nb), p.reshape(-1))
    xs = slice(0, g.nxf) if direction == "x" else slice(g.nxf, g.n_faces)
    other = slice(g.nxf, g.n_faces) if direction == "x" else slice(0, g.nxf)
    assert np.allclose(F[xs], 0.7 * 3.0 * g.hy if direction == "x" else 0.7 * 3.0 * g.hx, rtol=1e-12, atol=0)
    assert np.abs(F[other]).max() < 1e-12


def test_layered_piecewise_linear_exact():
    """kappa constant per column of cells, flow in x: the exact solution is
    continuous and piecewise linear with slope proportional to 1/kappa_i; it
    lies in V_h and SWIP (consistent) reproduces it."""
    nx, ny = 10, 4
    g = Grid(nx, ny, 1.0, 0.4)
    rng = np.random.default_rng(5)
    kcol = np.exp(rng.normal(0, 1.0, nx))
    perm = np.tile(kcol, ny)
    gam = np.full(g.n_cells, 1.3)
    bc, pD, vN, _ = default_bcs(nx, ny, p_left=2.0, p_right=-1.0)
    p = _solve(g, perm, gam, 40.0, bc, pD, vN).reshape(-1, 3)
    R = np.sum(g.hx / (1.3 * kcol))  # resistance per unit cross-section
    q = 3.0 / R
    xf = np.concatenate([[0.0], np.cumsum(np.full(nx, g.hx))])
    pf = 2.0 - np.concatenate([[0.0], np.cumsum(q * g.hx / (1.3 * kcol))])
    for e in range(g.n_cells):
        i = g.ci[e]
        slope = -q / (1.3 * kcol[i])
        assert abs(p[e, 0] - 0.5 * (pf[i] + pf[i + 1])) < 1e-11
        assert abs(p[e, 1] - slope * g.hx / 2) < 1e-11
        assert abs(p[e, 2]) < 1e-11
    F = face_fluxes(g, perm, gam, 40.0, bc, pD, vN, p.reshape(-1))
    assert np.allclose(F[:g.nxf], q * g.hy, rtol=1e-10)


def test_layered_tangential_exact():
    """kappa constant per row of cells, flow in x: p = 1 - x in every layer,
    the flux of each layer scales with its permeability."""
    nx, ny = 8, 6
    g = Grid(nx, ny, 1.0, 1.0)
    krow = np.exp(np.random.default_rng(7).normal(0, 1.5, ny))
    perm = np.repeat(krow, nx)
    gam = np.full(g.n_cells, 0.9)
    bc, pD, vN, _ = default_bcs(nx, ny)
    p = _solve(g, perm, gam, 20.0, bc, pD, vN).reshape(-1, 3)
    assert np.abs(p[:, 0] - (1 - g.xc)).max() < 1e-11
    assert np.abs(p[:, 2]).max() < 1e-11
    F = face_fluxes(g, perm, gam, 20.0, bc, pD, vN, p.reshape(-1))
    for j in range(ny):
        fx = F[j * (nx + 1):(j + 1) * (nx + 1)]
        assert np.allclose(fx, 0.9 * krow[j] * g.hy, rtol=1e-10)


def test_neumann_outflow_closed_form():
    """Reading R2: Dirichlet p_L on the left, outward flux v_N on the right:
    p = p_L - v_N x / (gamma kappa), and every face flux equals |f| v_N."""
    n = 10
    g = Grid(n, n, 2.0, 1.0)
    bc, pD, vN, _ = default_bcs(n, n, p_left=5.0, right="neumann", v_out=0.3)
    perm = np.full(g.n_cells, 2.0)
    gam = np.full(g.n_cells, 0.5)
    p = _solve(g, perm, gam, 20.0, bc, pD, vN).reshape(-1, 3)
    assert np.abs(p[:, 0] - (5.0 - 0.3 * g.xc / 1.0)).max() < 1e-11
    F = face_fluxes(g, perm, gam, 20.0, bc, pD, vN, p.reshape(-1))
    assert np.allclose(F[:g.nxf], 0.3 * g.hy, rtol=1e-10)


def test_manufactured_convergence():
    """Second-order L2 convergence to p = sin(pi x) sin(pi y) with source
    q1 = 2 pi^2 p, gamma kappa = 1 and p_D = 0 on all sides; a dropped term or a
    sign error in the face terms destroys the convergence."""
    errs = []
    for n in (16, 32, 64):
        g = Grid(n, n, 1.0, 1.0)
        nb = boundary_face_count(n, n)
        bc = np.ones(nb, dtype=np.int8)
        src = lambda x, y: 2 * np.pi ** 2 * np.sin(np.pi * x) * np.sin(np.pi * y)  # noqa: E731
        p = _solve(g, np.ones(g.n_cells), np.ones(g.n_cells), 10.0, bc, np.zeros(nb),
                   np.zeros(nb), source=src).reshape(-1, 3)
        xg, wg = np.polynomial.legendre.leggauss(4)
        err = 0.0
        for a, wa in zip(xg, wg):
            for b, wb in zip(xg, wg):
                x = g.xc + 0.5 * g.hx * a
                y = g.yc + 0.5 * g.hy * b
                v = g.basis_values(np.arange(g.n_cells), x, y)
                ph = np.einsum("ek,ek->e", v, p)
                err += np.sum(0.25 * g.vol * wa * wb * (ph - np.sin(np.pi * x) * np.sin(np.pi * y)) ** 2)
        errs.append(np.sqrt(err))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(rates > 1.85), (errs, rates)


def test_flux_local_conservation_mixed_bcs():
    """Definition 2 is locally conservative: per cell the outward fluxes sum
    to zero (heterogeneous kappa and mobility, Neumann outflow)."""
    prob = make_problem("paper_bc")
    m = FineModel.from_problem(prob)
    rng = np.random.default_rng(9)
    s = rng.uniform(0, 1, m.grid.n_cells)
    lam = m.mobility(s)
    p = m.solve_pressure(lam)
    F = m.fluxes(p, lam)
    # the per-cell sum cancels penalty terms of size ~ |K| |p|: bound by that scale
    K, _ = pressure_system(m.grid, m.perm, lam, m.c_pen, m.bc_type, m.p_D, m.v_N)
    scale = abs(K).sum(axis=1).max() * np.abs(p).max()
    assert np.abs(cell_outflows(m.grid, F)).max() <= 1e-13 * scale
    assert np.abs(cell_outflows(m.grid, F)).max() <= 1e-5 * np.abs(F).max()


def test_transpose_symmetry():
    """Swapping the roles of x and y (transposed permeability and boundary
    sides) transposes the solution: pins the x/y index handling."""
    nx, ny = 9, 7
    prob = make_problem("small")
    rng = np.random.default_rng(11)
    k = np.exp(rng.normal(0, 1, (ny, nx)))
    gam = rng.uniform(0.1, 1.0, (ny, nx))
    gA = Grid(nx, ny, 1.0, 0.8)
    bcA, pDA, vNA, _ = default_bcs(nx, ny, p_left=1.0, p_right=0.2)
    pA = _solve(gA, k.reshape(-1), gam.reshape(-1), 20.0, bcA, pDA, vNA).reshape(ny, nx, 3)
    gB = Grid(ny, nx, 0.8, 1.0)
    nb = boundary_face_count(ny, nx)
    bcB = np.zeros(nb, dtype=np.int8); pDB = np.zeros(nb)
    # A's left/right sides become B's bottom/top sides
    bcB[2 * nx:2 * nx + ny] = 1; pDB[2 * nx:2 * nx + ny] = 1.0
    bcB[2 * nx + ny:] = 1; pDB[2 * nx + ny:] = 0.2
    pB = _solve(gB, k.T.reshape(-1), gam.T.reshape(-1), 20.0, bcB, pDB, np.zeros(nb)).reshape(nx, ny, 3)
    assert np.allclose(pA[..., 0], pB[..., 0].T, atol=1e-12)
    assert np.allclose(pA[..., 1], pB[..., 2].T, atol=1e-12)
    assert np.allclose(pA[..., 2], pB[..., 1].T, atol=1e-12)


def test_consistency_sign_reading():
    """Reading R1: with the printed '+' sign on the consistency terms the
    linear closed form is lost; with '-' it is exact."""
    n = 6
    g = Grid(n, n, 1.0, 1.0)
    bc, pD, vN, _ = default_bcs(n, n)
    one = np.ones(g.n_cells)
    Kvp = bilinear(g, one, one, 20.0, bc, consistency=False)
    Kc = bilinear(g, one, one, 20.0, bc, volume=False, penalty=False)
    l_pen = linear(g, one, one, 20.0, bc, pD, vN, dirichlet_consistency=False)
    l_c = linear(g, one, one, 20.0, bc, pD, vN, dirichlet_penalty=False, neumann=False)
    exact = np.stack([1 - g.xc, np.full(g.n_cells, -g.hx / 2), np.zeros(g.n_cells)], 1).reshape(-1)
    p_minus = spla.spsolve((Kvp + Kc).tocsc(), l_pen + l_c)
    p_plus = spla.spsolve((Kvp - Kc).tocsc(), l_pen - l_c)
    assert np.abs(p_minus - exact).max() < 1e-12
    assert np.abs(p_plus - exact).max() > 1e-3
