"""Oracle: BAL camera model, residuals and Jacobians (Section 3.1, Eqs. 1-4).

Test infrastructure only (see ``oracle/__init__``).

The paper optimises d_p = 9 parameters per pose, extrinsics plus intrinsics,
on BAL data, but does not print the camera formula.  Reading used here: the
BAL model.  With c = (omega[3], t[3], f, k1, k2) and a landmark X,

    P   = R(omega) X + t          R(omega) by Rodrigues' formula
    p   = -(P_x, P_y) / P_z       (the camera looks down its -z axis)
    rho = 1 + k1 |p|^2 + k2 |p|^4
    pi  = f rho p
    r   = pi - m                  (m the measured pixel position)

Parameters are updated additively (x = x0 + dx, Eq. 3), so J_p is the
derivative with respect to omega itself.  For |omega| < 1e-8 the rotation is
taken to first order, R = I + [omega]_x.

Pins: J_p and J_l against central finite differences of ``residuals``;
R(omega) against rotation-matrix invariants and the closed form of a rotation
about a coordinate axis; the projection against the pinhole closed form.
"""
from __future__ import annotations

import numpy as np

SMALL_ANGLE = 1e-8


def _cross_matrix(v: np.ndarray) -> np.ndarray:
    """[v]_x for each row of v: (n, 3) -> (n, 3, 3)."""
    z = np.zeros(v.shape[0])
    return np.stack([
        np.stack([z, -v[:, 2], v[:, 1]], axis=1),
        np.stack([v[:, 2], z, -v[:, 0]], axis=1),
        np.stack([-v[:, 1], v[:, 0], z], axis=1),
    ], axis=1)


def rodrigues_coefficients(omega: np.ndarray):
    """theta = |omega| and the Rodrigues coefficients a = cos, b = sin/theta, c = (1 - cos)/theta^2."""
    theta = np.linalg.norm(omega, axis=1)
    small = theta < SMALL_ANGLE
    th = np.where(small, 1.0, theta)
    a = np.where(small, 1.0, np.cos(th))
    b = np.where(small, 1.0, np.sin(th) / th)
    c = np.where(small, 0.0, (1.0 - np.cos(th)) / (th * th))
    return theta, small, a, b, c


def rotation_matrix(omega: np.ndarray) -> np.ndarray:
    """R(omega) = a I + b [omega]_x + c omega omega^T, (n, 3) -> (n, 3, 3)."""
    _, _, a, b, c = rodrigues_coefficients(omega)
    eye = np.eye(3)[None]
    return (a[:, None, None] * eye + b[:, None, None] * _cross_matrix(omega)
            + c[:, None, None] * np.einsum("ni,nj->nij", omega, omega))


def project(cams: np.ndarray, pts: np.ndarray, obs_cam: np.ndarray, obs_pt: np.ndarray) -> np.ndarray:
    """pi(c_j, X_l) for every observation (j, l): (n_obs, 2)."""
    c = cams[obs_cam]
    X = pts[obs_pt]
    R = rotation_matrix(c[:, 0:3])
    P = np.einsum("nij,nj->ni", R, X) + c[:, 3:6]
    p = -P[:, 0:2] / P[:, 2:3]
    n2 = np.sum(p * p, axis=1)
    rho = 1.0 + c[:, 7] * n2 + c[:, 8] * n2 * n2
    return (c[:, 6] * rho)[:, None] * p


def residuals(cams, pts, obs_cam, obs_pt, obs_xy) -> np.ndarray:
    """r_i(x) = pi(c_j, X_l) - m_i, stacked (n_obs, 2) (Eq. 1)."""
    return project(cams, pts, obs_cam, obs_pt) - obs_xy


def cost(cams, pts, obs_cam, obs_pt, obs_xy) -> float:
    """F(x) = sum_i |r_i(x)|^2 (Eq. 1)."""
    r = residuals(cams, pts, obs_cam, obs_pt, obs_xy)
    return float(np.sum(r * r))


def jacobians(cams, pts, obs_cam, obs_pt):
    """Analytic J_p (n_obs, 2, 9) and J_l (n_obs, 2, 3) blocks of J = dr/dx (Eq. 4).

    Chain rule through P = R X + t, p = -P_xy / P_z, pi = f rho(p) p.  The
    rotation derivative differentiates R X = a X + b (omega x X) + c (omega . X) omega
    term by term, with d theta / d omega = omega / theta:
        da/domega = -b omega,  db/domega = (a - b)/theta^2 omega,
        dc/domega = (b - 2c)/theta^2 omega.
    """
    c = cams[obs_cam]
    X = pts[obs_pt]
    omega = c[:, 0:3]
    theta, small, a, b, cc = rodrigues_coefficients(omega)
    R = rotation_matrix(omega)
    P = np.einsum("nij,nj->ni", R, X) + c[:, 3:6]

    # dP/domega
    wx = np.cross(omega, X)
    wdotX = np.sum(omega * X, axis=1)
    th2 = np.where(small, 1.0, theta * theta)
    da = -b[:, None] * omega
    db = ((a - b) / th2)[:, None] * omega
    dc = ((b - 2.0 * cc) / th2)[:, None] * omega
    eye = np.eye(3)[None]
    dP_dw = (np.einsum("ni,nj->nij", X, da)
             + np.einsum("ni,nj->nij", wx, db)
             - b[:, None, None] * _cross_matrix(X)
             + np.einsum("ni,nj->nij", omega * wdotX[:, None], dc)
             + cc[:, None, None] * (wdotX[:, None, None] * eye + np.einsum("ni,nj->nij", omega, X)))
    dP_dw[small] = -_cross_matrix(X[small])

    # dp/dP
    iz = 1.0 / P[:, 2]
    p = -P[:, 0:2] * iz[:, None]
    dp_dP = np.zeros((P.shape[0], 2, 3))
    dp_dP[:, 0, 0] = -iz
    dp_dP[:, 1, 1] = -iz
    dp_dP[:, 0, 2] = P[:, 0] * iz * iz
    dp_dP[:, 1, 2] = P[:, 1] * iz * iz

    # dpi/dp and the intrinsics
    f, k1, k2 = c[:, 6], c[:, 7], c[:, 8]
    n2 = np.sum(p * p, axis=1)
    rho = 1.0 + k1 * n2 + k2 * n2 * n2
    drho_dn2 = k1 + 2.0 * k2 * n2
    dpi_dp = f[:, None, None] * (rho[:, None, None] * np.eye(2)[None]
                                 + 2.0 * drho_dn2[:, None, None] * np.einsum("ni,nj->nij", p, p))
    dpi_dP = np.einsum("nij,njk->nik", dpi_dp, dp_dP)

    Jp = np.empty((P.shape[0], 2, 9))
    Jp[:, :, 0:3] = np.einsum("nij,njk->nik", dpi_dP, dP_dw)
    Jp[:, :, 3:6] = dpi_dP
    Jp[:, :, 6] = rho[:, None] * p
    Jp[:, :, 7] = (f * n2)[:, None] * p
    Jp[:, :, 8] = (f * n2 * n2)[:, None] * p
    Jl = np.einsum("nij,njk->nik", dpi_dP, R)
    return Jp, Jl
