"""Oracle: linearised problem assembly, back-substitution and the LM loop (Sections 3.1, 4.1).

Test infrastructure only (see ``oracle/__init__``).

Back-substitution.  The paper prints dx_l = -V^{-1}(-b_l + W^T dx_p) (Eq. 15).
The second block row of Eq. 6, W^T dx_p + V_lambda dx_l = -b_l, gives
dx_l = -V_lambda^{-1}(b_l + W^T dx_p); that sign is the reading used.

LM loop (Section 4.1): lambda starts at 1e-4, at most 25 iterations, stop when
the relative decrease of F is below 1e-6.  The paper takes its lambda update
from another work and does not state it.  Reading used: accept a step when
F(x + dx) < F(x) and set lambda <- max(lambda / 10, 1e-12); otherwise reject
it and set lambda <- min(10 lambda, 1e16).

Pins: back-substitution against the landmark part of the dense solve of the
whole H; the LM claim that PCG and MCG give the same cost at every BA
iteration (Section 4.4) as a property test.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import camera, normal, schur, solvers


def measurements(scene) -> np.ndarray:
    """m = pi(c_true, X_true) + noise, with the oracle's own projection."""
    return camera.project(scene.cams_true, scene.pts_true, scene.obs_cam, scene.obs_pt) + scene.noise


@dataclass
class Linearised:
    r: np.ndarray
    Jp: np.ndarray
    Jl: np.ndarray
    ne: normal.NormalEquation
    S: object
    btilde: np.ndarray


def linearise(cams, pts, obs_cam, obs_pt, obs_xy, lam, damping="marquardt", with_schur=True) -> Linearised:
    """Residuals, Jacobians, normal equation and reduced camera system at (cams, pts)."""
    r = camera.residuals(cams, pts, obs_cam, obs_pt, obs_xy)
    Jp, Jl = camera.jacobians(cams, pts, obs_cam, obs_pt)
    ne = normal.normal_equation(Jp, Jl, r, obs_cam, obs_pt, cams.shape[0], pts.shape[0], lam, damping)
    S = bt = None
    if with_schur:
        S, bt = schur.schur_complement(ne, cams.shape[0], pts.shape[0])
    return Linearised(r, Jp, Jl, ne, S, bt)


def back_substitute(ne: normal.NormalEquation, dxp: np.ndarray, n_pts: int) -> np.ndarray:
    """dx_l = -V_lambda^{-1} (b_l + W^T dx_p), per landmark (Eq. 15, sign corrected)."""
    acc = ne.b_l.copy()
    contrib = np.einsum("nij,ni->nj", ne.W, dxp.reshape(-1, 9)[ne.obs_cam])
    np.add.at(acc, ne.obs_pt, contrib)
    return -np.linalg.solve(ne.V, acc[:, :, None])[:, :, 0]


@dataclass
class LMTrace:
    costs: list = field(default_factory=list)      # F after each iteration (accepted state)
    lambdas: list = field(default_factory=list)
    accepted: list = field(default_factory=list)
    solver_iters: list = field(default_factory=list)
    cams: np.ndarray | None = None
    pts: np.ndarray | None = None


def lm(cams, pts, obs_cam, obs_pt, obs_xy, solver="pcg", n_dirs=8, tau=3.0, lam0=1e-4,
       max_iters=25, ftol=1e-6, eps=1e-6, imax=1000, damping="marquardt") -> LMTrace:
    """Levenberg-Marquardt on F(x) with the reduced camera system solved by PCG or MCG."""
    cams = cams.copy()
    pts = pts.copy()
    lam = lam0
    F = camera.cost(cams, pts, obs_cam, obs_pt, obs_xy)
    tr = LMTrace(costs=[F])
    n_c, n_l = cams.shape[0], pts.shape[0]
    for _ in range(max_iters):
        lin = linearise(cams, pts, obs_cam, obs_pt, obs_xy, lam, damping)
        Dinv = solvers.block_jacobi_inverse(lin.S, n_c)
        if solver == "pcg":
            sol = solvers.pcg(lin.S, lin.btilde, Dinv, eps, imax)
        else:
            sol = solvers.mcg(lin.S, lin.btilde, Dinv, n_dirs, tau, eps, imax)
        dxl = back_substitute(lin.ne, sol.x, n_l)
        c_new = cams + sol.x.reshape(n_c, 9)
        p_new = pts + dxl
        F_new = camera.cost(c_new, p_new, obs_cam, obs_pt, obs_xy)
        tr.solver_iters.append(sol.iters)
        tr.lambdas.append(lam)
        if F_new < F:
            rel = (F - F_new) / F
            cams, pts, F = c_new, p_new, F_new
            lam = max(lam / 10.0, 1e-12)
            tr.accepted.append(True)
            tr.costs.append(F)
            if rel < ftol:
                break
        else:
            lam = min(lam * 10.0, 1e16)
            tr.accepted.append(False)
            tr.costs.append(F)
    tr.cams, tr.pts = cams, pts
    return tr
