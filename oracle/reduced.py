"""LRBMS online time step (Algorithm 3, step 5), FP64 on the CPU.

For n -> n+1 with saturation s^n:
  (a) fit theta(s^n) (Eq. leastSquaresFit) and assemble
      A = c + sum_q theta_q b_q, rhs = e + sum_q theta_q d_q (Eq. reducedSystem);
  (b) solve A x = rhs (a dense Cholesky factorisation; the system is SPD);
  (c) reconstruct p_h^r = sum_i x_i phi_i (step 5(b)) and the face fluxes of
      Definition 2 with lambda(s^n) (step 5(c), reading R7), or, as a
      variant, with the fitted mobility sum_q theta_q Lambda^q that the
      reduced pressure system itself uses (Section 4.4);
  (d) advance the saturation with Definition 3 (step 5(d)).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

from .impes import FineModel
from .offline import Offline
from .physics import total_mobility
from .transport import fv_update


def assemble(off: Offline, theta: np.ndarray):
    A = off.C + np.tensordot(theta, off.B, axes=1)
    rhs = off.e + theta @ off.d
    return A, rhs


def online_step(model: FineModel, off: Offline, s: np.ndarray, Phi_g=None, velocity: str = "state") -> dict:
    """One online step from saturation s. velocity: "state" (Definition 2
    with lambda(s^n), reading R7) or "fitted" (the fitted mobility)."""
    if Phi_g is None:
        Phi_g = off.extra["Phi_g"]
    lam = total_mobility(s, model.eta_w, model.eta_o, model.law)
    r = off.P @ lam
    theta = off.Gp @ r
    lam_fit = theta @ off.P
    A, rhs = assemble(off, theta)
    x = sla.cho_solve(sla.cho_factor(A), rhs)
    p = Phi_g @ x
    if velocity == "state":
        F = model.fluxes(p, lam)
    elif velocity == "fitted":
        F = model.fluxes(p, lam_fit)
    else:
        raise ValueError(velocity)
    dt = model.time_step(F)
    s_new, bout = fv_update(model.grid, s, F, model.poro, dt, model.s_D,
                            model.eta_w, model.eta_o, model.law)
    return dict(r=r, theta=theta, lam_fit=lam_fit, A=A, rhs=rhs, x=x, p=p, F=F, dt=dt,
                s=s_new, boundary_outflow=bout)


def online_run(model: FineModel, off: Offline, s0: np.ndarray, n_steps: int):
    s = np.array(s0, dtype=np.float64)
    hist = []
    for _ in range(n_steps):
        r = online_step(model, off, s)
        s = r["s"]
        hist.append(r)
    return s, hist


def online_step_dg(model: FineModel, off: Offline, c: np.ndarray, Phi_g=None) -> dict:
    """The online step with the piecewise-linear DG saturation and its limiter
    (Definition 3 with k = 1, Section 3.4): the fit, the reduced system and the
    fluxes take the mobility at the cell means c[:, 0]; the transport is
    oracle.transport_dg."""
    from .transport_dg import dg_step, dg_time_step, limit
    if Phi_g is None:
        Phi_g = off.extra["Phi_g"]
    s_mean = c[:, 0]
    lam = total_mobility(s_mean, model.eta_w, model.eta_o, model.law)
    r = off.P @ lam
    theta = off.Gp @ r
    A, rhs = assemble(off, theta)
    x = sla.cho_solve(sla.cho_factor(A), rhs)
    p = Phi_g @ x
    F = model.fluxes(p, lam)
    if model.dt_fixed is not None:
        dt = float(model.dt_fixed)
    else:
        dt = dg_time_step(model.grid, F, model.poro, model.Lf, model.cfl, model.dt_max)
    c_new, bout = dg_step(model.grid, c, F, model.poro, dt, model.s_D, model.eta_w, model.eta_o, model.law)
    c_lim, flagged = limit(model.grid, c_new, F, model.s_D)
    return dict(theta=theta, A=A, rhs=rhs, x=x, p=p, F=F, dt=dt, c_unlimited=c_new, c=c_lim,
                flagged=flagged, boundary_outflow=bout)
